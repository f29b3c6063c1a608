"""The synthetic workloads against the figures the paper prints (tests/golden/paper_workload.txt).

The paper prints no worked example with numerical results, so the fixture holds the workload
figures it does fix: the domain and fluid grids of the full and half-cube models (Section 4), the
membrane's length and mesh width (Section 4), and the time step with the 10 kHz run's length
(Section 5).  Every check measures the generated inputs themselves (marker positions, grid
sizes), not the constants they were built from, so a wrong helix pitch, grid size or spacing
fails here.  The bench's workloads depart from the paper in two figures, by choice: the membrane's
width profile and the half-cube's membrane (a shortened helix where the paper's is a flat spiral of
full length).  ``cochlea_halfcube_flat`` follows the paper in both and is checked against them.
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


def test_flat_halfcube_follows_the_paper():
    """Section 4's half-cube: 256 x 256 x 128 over 1 x 1 x 0.5 cm, the membrane flat (its spiral in
    one plane), 3.5 cm long, 150 -> 560 um wide, its mesh about half the fluid mesh; the wall tubes
    of neighbouring turns do not overlap; the structure is at rest in its reference shape."""
    from scipy.spatial import cKDTree

    import oracle
    p = synth.cochlea_halfcube_flat()
    st = p.structure
    check_grid(p, G["halfcube_grid"], G["halfcube_domain_cm"])
    nb, sh = st.n_membrane, st.sheets[0]
    X = st.X0
    assert np.ptp(X[2, :nb]) == 0.0                                  # flat
    length = np.linalg.norm(np.diff(centre_line(p), axis=1), axis=0).sum()
    assert length == pytest.approx(G["membrane_length_cm"], rel=2e-3)
    check_membrane_mesh(p)
    n1, n2 = sh.n1, sh.n2
    w_base = np.linalg.norm(X[:, n2 - 1] - X[:, 0])
    w_apex = np.linalg.norm(X[:, (n1 - 1) * n2 + n2 - 1] - X[:, (n1 - 1) * n2])
    np.testing.assert_allclose([w_base, w_apex], G["membrane_width_cm"], rtol=1e-12)
    # every wall marker is a tube radius or more from the whole centre line
    C = synth.flat_spiral_frame(np.arange(n1) * (G["membrane_length_cm"] / (n1 - 1)))[0]
    d = cKDTree(C.T).query(X[:, nb:].T)[0]
    assert d.min() >= synth.HALFCUBE_FLAT_TUBE * (1 - 1e-9)
    f = oracle.forces(oracle.Structure(st), np.zeros_like(X))
    assert np.abs(f).max() == 0.0
    assert abs(st.m - G["model_points"]) <= 0.1 * G["model_points"]   # 713,216 of about 750,000
