"""Stiffness gradient of the membrane misfit through the checkpointed reverse
sweep (paper_math_0301321_gb300.adjoint) against the oracle's reverse sweep
and against central finite differences of the FP64 forward.

The loss is the L2 misfit of the membrane's normal displacement over the
last `window` steps against a run with the unperturbed graded stiffness; the
stiffness is the graded profile times (1 + 0.1 xi), xi ~ N(0, 1) seeded.

For the finite-difference and oracle comparisons the small cochlea starts
from a membrane bump (three half-waves along its length) and carries 1e4
times the graded bending stiffness, so that over a dozen steps the
stiffness moves eta by about 1e-4 of itself: well above FP64 rounding, which
the misfit of two nearly equal runs would otherwise amplify.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.adjoint import MembraneRun, membrane_response, misfit

pytestmark = pytest.mark.gpu


def case(seed):
    p = synth.with_bend_scale(synth.cochlea_small(seed=seed), 1e4)
    return p, synth.membrane_bump(p, 1e-4, 3)


def gpu_grad(p, prec, b, n_steps, window, ckpt, D0=None, b_target=None):
    run = MembraneRun(p, prec=prec, n_steps=n_steps, window=window, ckpt_every=ckpt, D0=D0)
    with torch.no_grad():
        eta_t = run.forward(torch.tensor(p.structure.bend_b if b_target is None else b_target,
                                         dtype=torch.float64))
    theta = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    eta = membrane_response(theta, run)
    L = misfit(eta, eta_t)
    L.backward()
    g = theta.grad.detach().cpu().numpy().copy()
    run.close()
    return float(L.detach()), g, eta_t


def gpu_loss(p, prec, b, n_steps, window, eta_t, D0=None):
    run = MembraneRun(p, prec=prec, n_steps=n_steps, window=window, ckpt_every=n_steps, D0=D0)
    with torch.no_grad():
        L = float(misfit(run.forward(torch.tensor(b, dtype=torch.float64)), eta_t))
    run.close()
    return L


def oracle_sweep(p, b, n_steps, window, D0):
    """Loss and its stiffness gradient by the oracle: forward keeping every
    state, then oracle.adjoint_step backwards with the loss sensitivity
    added at each observed state."""
    g = p.grid
    M = p.structure.n_membrane
    n0 = p.structure.normal0[:, :M]
    first = n_steps - window + 1

    def run(bb):
        st = oracle.Structure(p.structure, bend_b=bb)
        D = np.asarray(D0, dtype=np.float64).copy()
        u = np.asarray(p.u, dtype=np.float64).copy()
        t = 0.0
        states = [(D, u, t)]
        for _ in range(n_steps):
            D, u, t = oracle.step(g, st, D, u, t, 1)
            states.append((D, u, t))
        eta = np.stack([(states[n][0][:, :M] * n0).sum(0) for n in range(first, n_steps + 1)])
        return st, states, eta

    _, _, eta_t = run(np.asarray(p.structure.bend_b))
    st, states, eta = run(b)
    L = ((eta - eta_t) ** 2).sum() / eta.size
    geta = 2.0 * (eta - eta_t) / eta.size
    lam_u = np.zeros_like(states[0][1])
    lam_D = np.zeros_like(states[0][0])
    grad = np.zeros(len(b))
    for n in range(n_steps - 1, -1, -1):
        j = n + 1 - first
        if j >= 0:
            lam_D[:, :M] += geta[j] * n0
        D, u, t = states[n]
        lam_u, lam_D, gb = oracle.adjoint_step(g, st, D, u, t, lam_u, lam_D)
        grad += gb
    return L, grad


@pytest.mark.parametrize("ckpt", [4, 5])
def test_gradient_matches_oracle_sweep_fp64(ib, ckpt):
    p, D0 = case(7)
    b = synth.perturbed_stiffness(p, 7)
    L, g, _ = gpu_grad(p, "fp64", b, 12, 6, ckpt, D0=D0)
    Lo, go = oracle_sweep(p, b, 12, 6, D0)
    # the misfit of two runs 1e-4 apart keeps about 12 - 4 digits of the
    # 1e-12 agreement of the two implementations' states
    assert abs(L - Lo) <= 1e-6 * abs(Lo)
    assert np.linalg.norm(g - go) <= 1e-6 * np.linalg.norm(go), (g, go)


def test_gradient_independent_of_checkpoint_spacing(ib):
    """Replays are bitwise deterministic, so the gradient does not depend on
    where the checkpoints are."""
    p, D0 = case(9)
    b = synth.perturbed_stiffness(p, 9)
    gs = [gpu_grad(p, "fp32", b, 10, 5, ck, D0=D0)[1] for ck in (3, 10, 1)]
    assert np.array_equal(gs[0], gs[1]) and np.array_equal(gs[0], gs[2])


def test_gradient_matches_fd_fp64(ib):
    """Central differences (h = 1e-4 relative) of the FP64 forward loss."""
    p, D0 = case(7)
    b = synth.perturbed_stiffness(p, 7)
    L, g, eta_t = gpu_grad(p, "fp64", b, 12, 6, 4, D0=D0)
    for s in range(len(b)):
        h = 1e-4 * b[s]
        bp, bm = b.copy(), b.copy()
        bp[s] += h
        bm[s] -= h
        fd = (gpu_loss(p, "fp64", bp, 12, 6, eta_t, D0) - gpu_loss(p, "fp64", bm, 12, 6, eta_t, D0)) / (2 * h)
        assert abs(fd - g[s]) <= 1e-4 * abs(g[s]), (s, fd, g[s])


def test_gradient_fp32_close_to_fp64(ib):
    p, D0 = case(7)
    b = synth.perturbed_stiffness(p, 7)
    _, g64, _ = gpu_grad(p, "fp64", b, 12, 6, 4, D0=D0)
    _, g32, _ = gpu_grad(p, "fp32", b, 12, 6, 4, D0=D0)
    assert np.linalg.norm(g32 - g64) <= 1e-2 * np.linalg.norm(g64), (g32, g64)


def test_gradient_workload_fd_eight_params(ib):
    """The 128^3 gradient workload (512x48 membrane, 64 stiffness segments,
    200k wall markers, 800 steps, snapshots every 40, misfit over the last
    200), started from a membrane bump with 1e4 times the graded bending
    stiffness (see the module docstring): the FP64 GPU gradient on 8 seeded
    parameters against FP64 central differences (h = 1e-4 relative) per
    parameter, and the FP32 GPU gradient norm-wise.  The FP32 bar is 5e-4:
    the misfit compares two forward runs whose membrane responses differ by
    about 1% of themselves, so the FP32 forward's per-step rounding reaches
    the misfit amplified about 100x (the FP32 loss is 8e-5 off the FP64
    loss; the FP32 gradient 1.7e-4 off the differences)."""
    p = synth.with_bend_scale(synth.cochlea128_adjoint(), 1e4)
    D0 = synth.membrane_bump(p, 1e-4, 3)
    b0 = np.asarray(p.structure.bend_b)
    b = synth.perturbed_stiffness(p, 5)
    idx = np.sort(np.minimum((synth.uniform(5, 81, 8) * len(b)).astype(int), len(b) - 1))
    grads = {}
    for prec in ("fp64", "fp32"):
        run = MembraneRun(p, prec=prec, n_steps=800, window=200, ckpt_every=40, D0=D0)
        with torch.no_grad():
            eta_t = run.forward(torch.tensor(b0))
        theta = torch.tensor(b, requires_grad=True)
        misfit(membrane_response(theta, run), eta_t).backward()
        grads[prec] = theta.grad.numpy()[idx]
        if prec == "fp64":
            fd = []
            for s in idx:
                h = 1e-4 * b[s]
                bp, bm = b.copy(), b.copy()
                bp[s] += h
                bm[s] -= h
                with torch.no_grad():
                    Lp = float(misfit(run.forward(torch.tensor(bp)), eta_t))
                    Lm = float(misfit(run.forward(torch.tensor(bm)), eta_t))
                fd.append((Lp - Lm) / (2 * h))
            fd = np.array(fd)
        run.close()
    assert np.all(np.abs(grads["fp64"] - fd) <= 1e-5 * np.abs(fd)), (grads["fp64"], fd)
    assert np.linalg.norm(grads["fp32"] - fd) <= 5e-4 * np.linalg.norm(fd), (grads["fp32"], fd)
