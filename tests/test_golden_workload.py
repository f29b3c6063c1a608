"""The synthetic workloads against the figures the paper prints (tests/golden/paper_workload.txt).

The paper prints no worked example with numerical results, so the fixture holds the workload
figures it does fix: the domain and fluid grids of the full and half-cube models (Section 4), the
membrane's length and mesh width (Section 4), and the time step with the 10 kHz run's length
(Section 5).  Every check measures the generated inputs themselves (marker positions, grid
sizes), not the constants they were built from, so a wrong helix pitch, grid size or spacing
fails here.  Two figures of the synthetic geometry depart from the paper by choice and are not
checked: the membrane's width profile and the half-cube's membrane (a shortened helix where the
paper's is a flat spiral of full length).
"""
import os

import numpy as np
import pytest

from paper_math_0301321_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_workload.txt")


def load_golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("|")[0].strip()
            if not line or line.startswith("#"):
                continue
            name, *rest = line.split()
            nums = [float(v) for v in rest]
            vals[name] = nums[0] if len(nums) == 1 else nums
    return vals


G = load_golden()


def centre_line(p):
    st = p.structure
    return st.X0[:, st.centerline]


def check_grid(p, grid, domain):
    g = p.grid
    assert tuple(g.n) == tuple(int(v) for v in grid)
    # one mesh width in every direction, and the grid spans the printed domain
    np.testing.assert_allclose([g.h * n for n in g.n], domain, rtol=1e-15)
    assert g.dt == G["dt_s"]
    X = p.structure.X0
    assert np.all(X >= 0.0)
    assert np.all(X < np.asarray(domain)[:, None])


def check_membrane_mesh(p):
    """Length-wise spacing of the membrane's markers about half the fluid mesh width."""
    seg = np.linalg.norm(np.diff(centre_line(p), axis=1), axis=0)
    ratio = seg / p.grid.h
    target = G["membrane_mesh_over_h"]
    assert np.all(np.abs(ratio - target) <= 0.25 * target), (ratio.min(), ratio.max())


def test_fixture_figures_agree():
    # the paper's run length and simulated time are consistent with its time step
    assert G["tone10k_steps"] * G["dt_s"] == pytest.approx(G["tone10k_time_s"], rel=1e-12)
    assert G["full_grid"] == [256.0, 256.0, 256.0]
    # the half-cube keeps the full model's mesh width: 1 cm / 256 in every direction
    hz = G["halfcube_domain_cm"][2] / G["halfcube_grid"][2]
    assert hz == G["full_domain_cm"][0] / G["full_grid"][0]


def test_full_cube_workload():
    p = synth.cochlea256()
    check_grid(p, G["full_grid"], G["full_domain_cm"])
    length = np.linalg.norm(np.diff(centre_line(p), axis=1), axis=0).sum()
    # the centre row is offset from the helix by 0.3% of the width: a few 1e-4 of the length
    assert length == pytest.approx(G["membrane_length_cm"], rel=2e-3)
    check_membrane_mesh(p)


def test_halfcube_workload():
    p = synth.cochlea_halfcube()
    check_grid(p, G["halfcube_grid"], G["halfcube_domain_cm"])
    check_membrane_mesh(p)


@pytest.mark.parametrize("make", [synth.cochlea128, synth.cochlea_windows, synth.cochlea128_adjoint])
def test_smaller_cochleas_keep_domain_and_time_step(make):
    p = make()
    n = p.grid.n
    check_grid(p, n, G["full_domain_cm"])


def test_tone_sweep_members_keep_domain_and_time_step():
    for p in synth.tone_sweep():
        check_grid(p, p.grid.n, G["full_domain_cm"])
