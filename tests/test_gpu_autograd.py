"""Gradient of the full objective through ism_gradient and the torch.autograd wrapper.

By Theorem 2 the library's dJ/du is beta_n times the sub-problem gradients at phi = phi^u; it must
equal the oracle's discrete gradient of J (trapezoid form) on the same seeded inputs.  Against
central differences of J itself it differs by exactly the trapezoid-vs-exact gap the oracle pins
(O(tau^2)); for the grid model the gradient is the exact reverse mode, so differences match it to
their own truncation error.
"""
import numpy as np
import pytest

import workloads as W
from oracle import gp_oracle as G
from oracle import ism_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _gp(n=64, Nt=120, N=6, T=1.5, seed=7):
    rng = np.random.default_rng(seed)
    psi_i, psi_f = W.gp_stationary_states(n, 20.0, -10.0, 1.0, dt=2e-3, steps=4000)
    return W.GPWorkload(name="gp", n=n, L=20.0, x_min=-10.0, g=1.0, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt, N=N,
                        u0=rng.uniform(-0.5, 0.5, Nt))


LINEAR = [
    ("spin16-fp64", W.with_random_target(W.config("spin16", Nt=300, N=5), 30), "fp64", 1e-10),
    ("rotor41-fp64", W.config("rotor41", Nt=800, N=8), "fp64", 1e-10),
    ("rotor41-mixed", W.config("rotor41", Nt=2000, N=16).with_(T=2000 * np.pi / 20000), "mixed", 1e-4),
    ("chain7-fp64", W.with_random_target(W.spin_chain(7, 91, T=1.0, Nt=150, N=5, u_amp=1.0), 31), "fp64", 1e-10),
    ("chain10-mixed", W.with_random_target(W.spin_chain(10, 92, T=0.4, Nt=2000, N=8, u_amp=1.0), 32), "mixed", 1e-4),
]


@pytest.mark.parametrize("name,w,prec,tol", LINEAR, ids=[c[0] for c in LINEAR])
def test_gradient_matches_oracle(P, name, w, prec, tol):
    g_o = O.global_gradient(w, w.u0)
    J_o, _ = O.objective(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, J = pl.gradient(w.u0)
    assert rel(g[0], g_o) <= tol, rel(g[0], g_o)
    assert abs(J[0] - J_o) <= (1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_gp_gradient_matches_oracle(P, prec, tol):
    w = _gp()
    g_o = G.global_gradient(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, J = pl.gradient(w.u0)
    assert rel(g[0], g_o) <= tol, rel(g[0], g_o)


def test_gradient_vs_central_differences_spin(P):
    """|g - FD| equals the oracle's trapezoid-vs-exact gap, up to the FD truncation error."""
    w = W.with_random_target(W.config("spin16", Nt=60, N=3), 33)
    u = w.u0
    with P.Plan(w, precision="fp64") as pl:
        g, _ = pl.gradient(u)
        h = 1e-5
        idx = [0, 7, 29, 59]
        U = np.repeat(u[None], 2 * len(idx), axis=0)
        for k, j in enumerate(idx):
            U[2 * k, j] += h
            U[2 * k + 1, j] -= h
    with P.Plan(w, precision="fp64", batch=U.shape[0]) as pl:
        Jp, _ = pl.evaluate(U)
    fd = np.array([(Jp[2 * k] - Jp[2 * k + 1]) / (2 * h) for k in range(len(idx))])
    gap = O.global_gradient(w, u)[idx] - O.exact_gradient(w, u)[idx]
    assert np.max(np.abs((g[0][idx] - fd) - gap)) <= 1e-8 * np.max(np.abs(fd)) + 1e-10


def test_gp_gradient_vs_central_differences(P):
    """Reverse mode of the split-step map: equal to differences of J to their truncation error."""
    w = _gp(Nt=40, N=4, T=0.8)
    with P.Plan(w, precision="fp64") as pl:
        g, _ = pl.gradient(w.u0)
    h = 1e-5
    idx = [0, 11, 39]
    U = np.repeat(w.u0[None], 2 * len(idx), axis=0)
    for k, j in enumerate(idx):
        U[2 * k, j] += h
        U[2 * k + 1, j] -= h
    with P.Plan(w, precision="fp64", batch=U.shape[0]) as pl:
        Jp, _ = pl.evaluate(U)
    fd = np.array([(Jp[2 * k] - Jp[2 * k + 1]) / (2 * h) for k in range(len(idx))])
    assert np.max(np.abs(g[0][idx] - fd)) <= 1e-8 * np.max(np.abs(fd))


def test_autograd_function(P):
    import torch

    from paper_1603_01237_gb300.autograd import objective

    w = W.config("rotor41", Nt=600, N=6)
    rng = np.random.default_rng(3)
    U = np.stack([w.u0, rng.uniform(-1, 1, w.Nt)])
    with P.Plan(w, precision="fp64", batch=2) as pl:
        u = torch.tensor(U, dtype=torch.float64, device="cuda", requires_grad=True)
        J = objective(u, pl)
        (J * torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda")).sum().backward()
        g, Jr = pl.gradient(U)
    assert np.array_equal(J.detach().cpu().numpy(), Jr)
    assert np.allclose(u.grad.cpu().numpy(), np.stack([g[0], -2.0 * g[1]]), rtol=0, atol=0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-4)])
def test_gp_autograd_function_vs_central_differences(P, prec, tol):
    """The condensate's adjoint through torch.autograd: J = objective(u, plan) on a 64-point grid,
    J.backward() runs ism_gradient (exact reverse mode of the split-step map), and u.grad equals central
    differences of J (FP64 plan, h = 1e-5) to their truncation error, and the FP64 oracle's
    reverse-mode gradient at the stated tolerance."""
    import torch

    from paper_1603_01237_gb300.autograd import objective

    w = _gp(Nt=40, N=4, T=0.8)
    rng = np.random.default_rng(5)
    U = np.stack([w.u0, rng.uniform(-0.5, 0.5, w.Nt)])
    with P.Plan(w, precision=prec, batch=2) as pl:
        u = torch.tensor(U, dtype=torch.float64, device="cuda", requires_grad=True)
        J = objective(u, pl)
        J.sum().backward()
        g = u.grad.cpu().numpy()
    h = 1e-5
    idx = [0, 17, 39]
    for b in range(2):
        V = np.repeat(U[b][None], 2 * len(idx), axis=0)
        for k, j in enumerate(idx):
            V[2 * k, j] += h
            V[2 * k + 1, j] -= h
        with P.Plan(w, precision="fp64", batch=V.shape[0]) as pl:
            Jp, _ = pl.evaluate(V)
        fd = np.array([(Jp[2 * k] - Jp[2 * k + 1]) / (2 * h) for k in range(len(idx))])
        assert np.max(np.abs(g[b][idx] - fd)) <= max(tol, 1e-8) * np.max(np.abs(fd)), (b, g[b][idx], fd)
        g_o = G.global_gradient(w, U[b])
        assert rel(g[b], g_o) <= (1e-10 if prec == "fp64" else tol), rel(g[b], g_o)
