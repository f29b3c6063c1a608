"""GPU parity of the reverse step (ib_adjoint_step) against the oracle's
reverse step, which the CPU tests pin to finite differences of the forward
oracle.

Bars: FP64 contexts within 1e-12 relative (norm-wise), FP32 contexts within
2e-5 relative.  The marker sensitivity is compared without its identity part
(lam_D^n - lam_D^{n+1}), which is what the step actually computes.  FP32
cases hand the oracle the FP32-rounded state and inputs, so both sides start
from the same numbers.
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def rounded(a, prec):
    return np.asarray(a, np.float32).astype(np.float64) if prec == "fp32" else np.asarray(a, np.float64)


def state(p, seed, u_scale=20.0):
    """Uniform flow plus a perturbation of 0.3 of its smallest component (no
    velocity component near zero, so both sides take the same upwind
    branches), small random displacements, and a time inside the forcing."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = p.grid.n
    mean = u_scale * np.array([1.0, -0.8, 0.9])
    u = mean[:, None, None, None] + 0.24 * u_scale * (2 * rng.random((3, nz, ny, nx)) - 1)
    D = 1e-4 * rng.standard_normal(p.structure.X0.shape)
    return u, D, 1.3e-4, rng


def gpu_adjoint(p, prec, u, D, t, lam_u, lam_D, u_np1=None, device=True, bend_b=None):
    ctx = Context(p.grid, prec=prec, device=device)
    ctx.set_structure(p.structure, bend_b=bend_b)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    nseg = len(p.structure.bend_b)
    gb = torch.zeros(nseg, dtype=torch.float64, device="cuda") if device else np.zeros(nseg)
    luo, lDo = ctx.adjoint_step(lam_u, lam_D, u_np1=u_np1, grad_b=gb)
    out = host(luo).astype(np.float64), host(lDo), host(gb).copy()
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["u", "D"])
def test_adjoint_step_matches_oracle(ib, prec, which):
    p = synth.cochlea_small(seed=7)
    u, D, t, rng = state(p, 41)
    u, D = rounded(u, prec), rounded(D, prec)
    lam_u = rng.standard_normal(u.shape) if which == "u" else np.zeros(u.shape)
    lam_D = rng.standard_normal(D.shape) if which == "D" else np.zeros(D.shape)
    lam_u = rounded(lam_u, prec)
    lam_D = rounded(lam_D, prec)
    st = oracle.Structure(p.structure)
    lu0, lD0, gb = oracle.adjoint_step(p.grid, st, D, u, t, lam_u, lam_D)
    luo, lDo, ggb = gpu_adjoint(p, prec, u, D, t, lam_u, lam_D)
    tol = TOL[prec]
    assert rel(luo, lu0) <= tol, rel(luo, lu0)
    assert rel(lDo - lam_D, lD0 - lam_D) <= tol, rel(lDo - lam_D, lD0 - lam_D)
    assert rel(ggb, gb) <= tol, (ggb, gb)


def test_adjoint_step_sphere_fp64(ib):
    """Springs only (no bending, tethers or forcing), 32^3 icosphere."""
    p = synth.sphere32()
    u, D, _, rng = state(p, 42, 5.0)
    D = 1e-3 * rng.standard_normal(D.shape)
    lam_u = rng.standard_normal(u.shape)
    lam_D = rng.standard_normal(D.shape)
    st = oracle.Structure(p.structure)
    lu0, lD0, _ = oracle.adjoint_step(p.grid, st, D, u, 0.0, lam_u, lam_D)
    luo, lDo, _ = gpu_adjoint(p, "fp64", u, D, 0.0, lam_u, lam_D)
    assert rel(luo, lu0) <= 1e-12
    assert rel(lDo - lam_D, lD0 - lam_D) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_given_u_np1_is_bitwise_the_recompute(ib, prec):
    """Passing u^{n+1} from ib_step gives bitwise the same result as letting
    the reverse step recompute it, and two runs are bitwise identical."""
    p = synth.cochlea_small(seed=9)
    u, D, t, rng = state(p, 43)
    lam_u = rng.standard_normal(u.shape)
    lam_D = rng.standard_normal(D.shape)
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    ctx.step(1)
    u1, _, _ = ctx.get_state()
    u1 = u1.clone()
    ctx.close()
    a = gpu_adjoint(p, prec, u, D, t, lam_u, lam_D)
    b = gpu_adjoint(p, prec, u, D, t, lam_u, lam_D, u_np1=u1)
    c = gpu_adjoint(p, prec, u, D, t, lam_u, lam_D)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        assert np.array_equal(x, z)


def test_adjoint_host_pointers_match_device(ib):
    p = synth.cochlea_small(seed=7)
    u, D, t, rng = state(p, 44)
    lam_u = rng.standard_normal(u.shape)
    lam_D = rng.standard_normal(D.shape)
    a = gpu_adjoint(p, "fp64", u, D, t, lam_u, lam_D, device=True)
    b = gpu_adjoint(p, "fp64", u, D, t, lam_u, lam_D, device=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_adjoint_two_steps_chain_fp64(ib):
    """Two reverse steps, each about its own forward state, against the
    oracle's two reverse steps; the stiffness gradient accumulates."""
    p = synth.cochlea_small(seed=8)
    u0, D0, t0, rng = state(p, 45)
    st = oracle.Structure(p.structure)
    D1, u1, t1 = oracle.step(p.grid, st, D0, u0, t0, 1)
    lam_u = rng.standard_normal(u0.shape)
    lam_D = rng.standard_normal(D0.shape)
    a1 = oracle.adjoint_step(p.grid, st, D1, u1, t1, lam_u, lam_D)
    a0 = oracle.adjoint_step(p.grid, st, D0, u0, t0, a1[0], a1[1])

    ctx = Context(p.grid, prec="fp64")
    ctx.set_structure(p.structure)
    gb = torch.zeros(len(p.structure.bend_b), dtype=torch.float64, device="cuda")
    ctx.set_state(u1, None, t1)
    ctx.set_displacement(D1)
    lu, lD = ctx.adjoint_step(lam_u, lam_D, grad_b=gb)
    ctx.set_state(u0, None, t0)
    ctx.set_displacement(D0)
    lu, lD = ctx.adjoint_step(lu, lD, grad_b=gb, out=(lu, lD))     # in place
    assert rel(host(lu), a0[0]) <= 1e-12
    assert rel(host(lD) - lam_D, a0[1] - lam_D) <= 1e-12
    assert rel(host(gb), a0[2] + a1[2]) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_set_bend_stiffness_matches_structure(ib, prec):
    """A step after ib_set_bend_stiffness equals the oracle's step with that
    stiffness, and equals setting the structure with it (bitwise)."""
    p = synth.cochlea_small(seed=7)
    u, D, t, rng = state(p, 46)
    u, D = rounded(u, prec), rounded(D, prec)
    b = np.asarray(p.structure.bend_b) * (1 + 0.3 * rng.standard_normal(len(p.structure.bend_b)))
    outs = []
    for mode in ("update", "structure"):
        ctx = Context(p.grid, prec=prec)
        if mode == "update":
            ctx.set_structure(p.structure)
            ctx.set_bend_stiffness(b)
        else:
            ctx.set_structure(p.structure, bend_b=b)
        ctx.set_state(u, None, t)
        ctx.set_displacement(D)
        ctx.step(1)
        uu, _, _ = ctx.get_state()
        outs.append((host(uu).astype(np.float64), host(ctx.get_displacement())))
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    Do, uo, _ = oracle.step(p.grid, oracle.Structure(p.structure, bend_b=b), D, u, t, 1)
    tol = TOL[prec]
    assert rel(outs[0][0], uo) <= tol
    assert rel(outs[0][1] - D, Do - D) <= (tol if prec == "fp64" else 1e-4)


def test_adjoint_rejects_null_inputs(ib):
    p = synth.cochlea_small(seed=7)
    ctx = Context(p.grid, prec="fp64")
    ctx.set_structure(p.structure)
    import ctypes as C
    from paper_math_0301321_gb300.binding import IB_ERR_ARG
    st = ctx.lib.ib_adjoint_step(ctx.h, None, None, None, None, None, None)
    assert st == IB_ERR_ARG
