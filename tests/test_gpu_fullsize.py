"""Full-size parity: one step of the benchmark workload (256^3, 993,216
markers) and of the 128^3 cochlea, as ib_step runs it (the captured graph),
against one oracle step from the same state.

The state is the workload's structure with nanometre displacements (a
membrane bump of 1e-7 cm plus 2e-8 cm of seeded noise on every marker) and a
smooth seeded velocity field of 0.1 cm/s, so that every force law, both
upwind branches, spreading, the solve, the body force and interpolation all
contribute.  Bars: FP64 1e-12, FP32 2e-5 (norm-wise), on the velocity and on
the displacement increment of the step; the same bars on the largest element
error relative to the field's largest element, and on the velocity's
norm-wise error within every 8^3 tile, so that a wrong value confined to a
few cells of the grid cannot hide under the whole-field norm.  The step's
own bin sort (keys from the state X0 + D, markers in tile order) equals the
oracle's bit for bit in both precisions.
"""
import numpy as np
import pytest

import oracle
from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Context

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state(p, seed):
    D = synth.membrane_bump(p, 1e-7, 3) + 2e-8 * synth.normal(seed, 61, 3 * p.structure.m).reshape(3, -1)
    u = synth.random_velocity(seed, p.grid.n, amp=0.1, modes=8)
    return D, u, 2.0e-5


def max_rel(a, b):
    """Largest element error relative to the largest element of b."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def worst_tile(a, b, tile=8):
    """Largest norm-wise error of a vector field [3][z][y][x] over the tiles."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    _, nz, ny, nx = b.shape
    shp = (3, nz // tile, tile, ny // tile, tile, nx // tile, tile)
    num = ((a - b).reshape(shp) ** 2).sum(axis=(0, 2, 4, 6))
    den = (b.reshape(shp) ** 2).sum(axis=(0, 2, 4, 6))
    return float(np.sqrt(num / den).max())


def gpu_step(p, prec, D, u, t, order=False):
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    ctx.step(1)
    uu, _, tt = ctx.get_state()
    DD = ctx.get_displacement()
    out = uu.cpu().numpy().astype(np.float64), DD.cpu().numpy(), tt
    if order:
        out = out + tuple(o.cpu().numpy() for o in ctx.get_bin_order())
    ctx.close()
    return out


def oracle_order(p, D, internal):
    """The oracle's bin sort of X0 + D with markers numbered as the context
    numbers them internally, returned in the caller's numbering."""
    X = np.asarray(p.structure.X0, np.float64) + D
    ko, po = oracle.bin_sort(p.grid, X[:, internal])
    key = np.empty_like(ko)
    key[internal] = ko
    return key, internal[po]


@pytest.mark.parametrize("name", ["cochlea128", "cochlea256"])
def test_one_full_size_step_matches_oracle(ib, name):
    p = getattr(synth, name)()
    D, u, t = state(p, 17)
    st = oracle.Structure(p.structure)
    for prec in ("fp64", "fp32"):
        # both sides start from the state the context actually holds
        Ds = np.asarray(D, np.float32).astype(np.float64) if prec == "fp32" else D
        us = np.asarray(u, np.float32).astype(np.float64) if prec == "fp32" else u
        Do, uo, to = oracle.step(p.grid, st, Ds, us, t, 1)
        ug, Dg, tg, key, perm, internal = gpu_step(p, prec, Ds, us, t, order=True)
        assert abs(tg - to) <= 1e-15
        assert rel(ug, uo) <= TOL[prec], (prec, rel(ug, uo))
        assert rel(Dg - Ds, Do - Ds) <= TOL[prec], (prec, rel(Dg - Ds, Do - Ds))
        assert max_rel(ug, uo) <= TOL[prec], (prec, max_rel(ug, uo))
        assert max_rel(Dg - Ds, Do - Ds) <= TOL[prec], (prec, max_rel(Dg - Ds, Do - Ds))
        assert worst_tile(ug, uo) <= TOL[prec], (prec, worst_tile(ug, uo))
        assert sorted(internal.tolist()) == list(range(p.structure.m))
        ko, po = oracle_order(p, Ds, internal)
        assert np.array_equal(key, ko), (prec, int((key != ko).sum()))
        assert np.array_equal(perm, po), (prec, int((perm != po).sum()))


def test_cochlea128_fp32_step_at_steps_1_10_100(ib):
    """The 128^3 cochlea from rest: the FP64 GPU path (equal to the oracle to
    1e-12, tested above and in test_gpu_parity) provides the states after 0,
    9 and 99 steps; from each, one FP32 step against one oracle step (step 1,
    10 and 100 of the run), per-step bar 2e-5 on u and on the displacement
    increment."""
    p = synth.cochlea128()
    st = oracle.Structure(p.structure)
    c64 = Context(p.grid, prec="fp64")
    c64.set_structure(p.structure)
    c64.set_state(p.u, None, 0.0)
    c64.set_displacement(np.zeros_like(p.structure.X0))
    done = 0
    for k in (1, 10, 100):
        c64.step(k - 1 - done)
        done = k - 1
        u, _, t = c64.get_state()
        D = c64.get_displacement().cpu().numpy()
        u = u.cpu().numpy()
        Ds = np.asarray(D, np.float32).astype(np.float64)
        us = np.asarray(u, np.float32).astype(np.float64)
        Do, uo, _ = oracle.step(p.grid, st, Ds, us, t, 1)
        ug, Dg, _ = gpu_step(p, "fp32", Ds, us, t)
        assert rel(ug, uo) <= TOL["fp32"], (k, rel(ug, uo))
        dD = Do - Ds
        if np.abs(dD).max() > 0:
            assert rel(Dg - Ds, dD) <= TOL["fp32"], (k, rel(Dg - Ds, dD))
    c64.close()
