"""The tensor-core y passes (IB_FP32_TCFFT): the fluid solve of Eqs.
(discreteNS1)-(discreteNS2) with the y FFTs as split-BF16 DFT products
against the FP64 oracle's solve, and one step of the small cochlea against
the oracle's step.

Bar: the BF16 split represents each operand to about 2^-16 of itself (the
high part to 2^-8, the rounded remainder to 2^-8 of that), so each radix-16
stage's outputs carry about 2^-16 relative error; two stages per y pass, two
y passes per solve: 2e-4 relative (norm-wise) bounds it with margin.  The
measured errors are printed."""
import numpy as np
import pytest

import oracle
from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Context

pytestmark = pytest.mark.gpu

TOL_TC = 2e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Grid:
    def __init__(self, n, h=1.0 / 256, rho=1.0, mu=0.02, dt=1e-6):
        self.n, self.h, self.rho, self.mu, self.dt = tuple(n), h, rho, mu, dt


@pytest.mark.parametrize("n", [(32, 256, 32), (64, 256, 96)])
def test_tcfft_solve_matches_oracle(ib, n):
    g = Grid(n)
    u = synth.random_velocity(3, n, amp=1.0, modes=6, noise=0.1)
    F = 1e3 * synth.random_velocity(4, n, amp=1.0, modes=5, noise=0.2)
    u = np.asarray(u, np.float32).astype(np.float64)
    F = np.asarray(F, np.float32).astype(np.float64)
    uo = oracle.fluid_solve(g, u, F)
    out = {}
    for prec in ("fp32", "fp32_tcfft"):
        ctx = Context(g, prec=prec)
        out[prec] = ctx.fluid_solve(u, F).cpu().numpy().astype(np.float64)
        ctx.close()
    e32, etc = rel(out["fp32"], uo), rel(out["fp32_tcfft"], uo)
    print(f"solve {n}: FP32 {e32:.2e}, split-BF16 tensor-core y passes {etc:.2e}")
    assert e32 <= 2e-5
    assert etc <= TOL_TC, etc


def test_tcfft_step_matches_oracle(ib):
    q = synth.sphere_problem(seed=1, n=32)
    # a grid with a 256-long y axis around the same sphere
    g = Grid((32, 256, 32), h=q.grid.h, rho=q.grid.rho, mu=q.grid.mu, dt=q.grid.dt)
    st = q.structure
    u = np.zeros((3, 32, 256, 32))
    st_o = oracle.Structure(st)
    Do, uo, _ = oracle.step(g, st_o, np.zeros_like(st.X0), u, 0.0, 2)
    ctx = Context(g, prec="fp32_tcfft")
    ctx.set_structure(st)
    ctx.set_state(u, None, 0.0)
    ctx.step(2)
    ug, _, _ = ctx.get_state()
    Dg = ctx.get_displacement().cpu().numpy()
    ctx.close()
    eu, ed = rel(ug.cpu().numpy(), uo), rel(Dg, Do)
    print(f"two steps, sphere on 32x256x32: u {eu:.2e}, D {ed:.2e}")
    assert eu <= TOL_TC and ed <= TOL_TC, (eu, ed)
