"""The allocation-free entry point ism_subinterval_grad_noalloc.

It serves callers that cannot allocate device memory themselves (code inside another framework's
memory pool, allocation-free real-time loops, fixed device-memory budgets): no plan, no cudaMalloc,
all scratch in one static device array.  Each test compares it, through the C ABI, with the planned
entry point ism_subinterval_grad on the same device inputs, for two calls in a row with different
inputs, so a stale scratch array from the previous call would show.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    import paper_1603_01237_gb300 as P
    from paper_1603_01237_gb300 import abi

    return P, abi, torch


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    ("rotor41-mixed", W.config("rotor41", Nt=2000, N=16), "mixed", 1e-4),
    ("spin16-fp64", W.config("spin16", Nt=400, N=7).with_(u0=np.random.default_rng(3).uniform(-1.5, 1.5, 400)), "fp64", 1e-10),
    ("dense24-obs-fp64", W.random_dense(24, 81, T=2.0, Nt=300, N=9, objective="observable"), "fp64", 1e-10),
]


@pytest.mark.parametrize("name,w,prec,tol", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_planned_entry_point(env, name, w, prec, tol):
    P, abi, torch = env
    rng = np.random.default_rng(11)
    u_list = [w.u0, w.u0 + rng.uniform(-0.2, 0.2, w.Nt)]
    with P.Plan(w, precision=prec) as plan:
        for u in u_list:                                  # two calls in a row, different inputs
            phi = plan.intermediate_states(u)
            phi_d = torch.tensor(phi.view(np.float64), device="cuda")
            u_d = torch.tensor(u, dtype=torch.float64, device="cuda").reshape(1, -1)
            g_ref = torch.empty((1, w.Nt), dtype=torch.float64, device="cuda")
            J_ref = torch.empty((1, w.N), dtype=torch.float64, device="cuda")
            plan.ism_subinterval_grad(phi_d, u_d, g_ref, J_ref)
            g = torch.full((1, w.Nt), float("nan"), dtype=torch.float64, device="cuda")
            J = torch.full((1, w.N), float("nan"), dtype=torch.float64, device="cuda")
            abi.subinterval_grad_noalloc(w, prec, phi_d, u_d, g, J)
            a, b = g.cpu().numpy(), g_ref.cpu().numpy()
            assert np.isfinite(a).all()
            assert _rel(a, b) <= tol, _rel(a, b)
            assert np.max(np.abs(J.cpu().numpy() - J_ref.cpu().numpy())) <= tol * max(1.0, np.abs(J_ref.cpu().numpy()).max())


def test_noalloc_rejects_oversize_and_host_buffers(env):
    P, abi, torch = env
    w = W.config("rotor41", Nt=2000, N=16)
    big = w.with_(Nt=200000, N=16, u0=np.zeros(200000), alpha=None)   # trajectory > static scratch
    dev = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")   # noqa: E731
    with pytest.raises(abi.IsmError) as ei:
        abi.subinterval_grad_noalloc(big, "fp64", dev(2 * 17 * 41), dev(200000), dev(200000), None)
    assert ei.value.status == abi.ISM_EINVAL and "bytes of scratch" in str(ei.value)
    with pytest.raises(abi.IsmError) as ei:
        abi.subinterval_grad_noalloc(w, "mixed", np.zeros(2 * 17 * 41), np.zeros(2000), np.zeros(2000), None)
    assert ei.value.status == abi.ISM_EINVAL
