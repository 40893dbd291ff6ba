"""The allocation-free entry point ism_subinterval_grad_noalloc.

It serves callers that cannot allocate device memory themselves (code inside another framework's
memory pool, allocation-free real-time loops, fixed device-memory budgets): no plan, no cudaMalloc,
all scratch in one static device array.  It launches the same kernels as the planned entry point
ism_subinterval_grad on the same inputs, so each test requires its results to equal the planned
call's bit for bit, and to match the FP64 oracle's sub-problem gradients at the parity tolerances;
two calls in a row with different inputs show that a stale scratch array from the previous call
changes nothing.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ism_oracle as O

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


# (name, workload, precision, gradient relative L2 vs the oracle, J_n absolute vs the oracle, batch)
CASES = [
    ("rotor41-mixed", W.config("rotor41", Nt=2000, N=16), "mixed", 1e-4, 1e-5, 1),
    ("spin16-fp64", W.config("spin16", Nt=400, N=7).with_(u0=np.random.default_rng(3).uniform(-1.5, 1.5, 400)),
     "fp64", 1e-10, 1e-12, 1),
    ("dense24-obs-fp64", W.random_dense(24, 81, T=2.0, Nt=300, N=9, objective="observable"), "fp64", 1e-10, 1e-12, 1),
    ("rotor41-mixed-batch3", W.config("rotor41", Nt=1203, N=11), "mixed", 1e-4, 1e-5, 3),
]


@pytest.mark.parametrize("name,w,prec,gtol,jtol,batch", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_planned_entry_point_and_oracle(env, name, w, prec, gtol, jtol, batch):
    P, abi, torch = env
    rng = np.random.default_rng(11)
    B, Nt, N = batch, w.Nt, w.N
    for call in range(2):                               # two calls in a row, different inputs
        # different controls per problem (and per call); phi = phi^u of each problem's controls
        u = np.stack([w.u0 + (0 if (call == 0 and b == 0) else rng.uniform(-0.2, 0.2, Nt)) for b in range(B)])
        phi = np.stack([O.intermediate_states(w, u[b]) for b in range(B)])
        phi_d = torch.tensor(phi.view(np.float64), device="cuda")
        u_d = torch.tensor(u, dtype=torch.float64, device="cuda")
        with P.Plan(w, precision=prec, batch=B) as plan:
            g_ref = torch.empty((B, Nt), dtype=torch.float64, device="cuda")
            J_ref = torch.empty((B, N), dtype=torch.float64, device="cuda")
            plan.ism_subinterval_grad(phi_d, u_d, g_ref, J_ref)
        g = torch.full((B, Nt), float("nan"), dtype=torch.float64, device="cuda")
        J = torch.full((B, N), float("nan"), dtype=torch.float64, device="cuda")
        abi.subinterval_grad_noalloc(w, prec, phi_d, u_d, g, J, batch=B)
        g, J, g_ref, J_ref = g.cpu().numpy(), J.cpu().numpy(), g_ref.cpu().numpy(), J_ref.cpu().numpy()
        assert np.array_equal(g, g_ref), np.max(np.abs(g - g_ref))      # the same kernels on the same inputs
        assert np.array_equal(J, J_ref), np.max(np.abs(J - J_ref))
        for b in range(B):
            g_o, Jn_o = O.subinterval_all(w, phi[b], u[b])
            assert _rel(g[b], g_o) <= gtol, (b, _rel(g[b], g_o))
            assert np.max(np.abs(J[b] - Jn_o)) <= jtol * max(1.0, np.abs(Jn_o).max())


def test_noalloc_rejects_oversize_host_buffers_and_nonfinite(env):
    P, abi, torch = env
    w = W.config("rotor41", Nt=2000, N=16)
    dev = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")   # noqa: E731
    # 256 problems of 50000 steps: the per-step overlaps alone exceed the static scratch
    big = w.with_(Nt=50000, N=16, u0=np.zeros(50000), alpha=None)
    with pytest.raises(abi.IsmError) as ei:
        abi.subinterval_grad_noalloc(big, "fp64", dev(256 * 2 * 17 * 41), dev(256 * 50000), dev(256 * 50000), None,
                                     batch=256)
    assert ei.value.status == abi.ISM_EINVAL and "bytes of scratch" in str(ei.value)
    with pytest.raises(abi.IsmError) as ei:
        abi.subinterval_grad_noalloc(w, "mixed", np.zeros(2 * 17 * 41), np.zeros(2000), np.zeros(2000), None)
    assert ei.value.status == abi.ISM_EINVAL
    # a NaN control: ISM_ENONFINITE (not a NaN gradient with ISM_OK)
    phi = O.intermediate_states(w, w.u0)
    u = w.u0.copy()
    u[1234] = np.nan
    phi_d = torch.tensor(phi.view(np.float64).ravel(), device="cuda")
    with pytest.raises(abi.IsmError) as ei:
        abi.subinterval_grad_noalloc(w, "mixed", phi_d, torch.tensor(u, device="cuda"), dev(2000), dev(16))
    assert ei.value.status == abi.ISM_ENONFINITE
    # the scratch is usable again after the refused calls
    g = dev(2000)
    abi.subinterval_grad_noalloc(w, "mixed", phi_d, torch.tensor(w.u0, device="cuda"), g, None)
    g_o, _ = O.subinterval_all(w, phi, w.u0)
    assert _rel(g.cpu().numpy(), g_o) <= 1e-4
