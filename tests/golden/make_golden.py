"""Write the stored expected values used by the full-size GPU parity tests.

Every number here comes from the FP64 oracles (oracle/ism_oracle.py, oracle/gp_oracle.py) run on
the seeded workloads of the `workloads` package; nothing is read from the CUDA path.

    python tests/golden/make_golden.py rotor41      # ~15-30 min on one core
    python tests/golden/make_golden.py gp512        # ~2-4 min
    python tests/golden/make_golden.py ising1024    # ~15-25 min
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import gp_oracle as G  # noqa: E402
from oracle import ism_oracle as O  # noqa: E402


def rotor41():
    """Full rigid-rotor benchmark problem: d=41, Nt=20000, N=128, 50 iterations, rho=1.  With one
    local step the iterates do not depend on N (Theorem 2), so the history holds for N = 16, 64, 128."""
    w = W.config("rotor41")
    t0 = time.time()
    u, J, F, E = O.ism_solve(w, w.u0, w.iters, w.rho)
    idx = np.arange(0, w.Nt, 97)
    return {
        "workload": "rotor41", "d": w.d, "Nt": w.Nt, "N": w.N, "iters": w.iters, "rho": w.rho,
        "source": "oracle.ism_oracle.ism_solve (FP64, exact step exponentials)",
        "J_hist": J.tolist(), "F_hist": F.tolist(), "err_hist": E.tolist(),
        "u_final_idx": idx.tolist(), "u_final": u[idx].tolist(),
        "oracle_seconds": time.time() - t0,
    }


def rotor41_first_gradient():
    """Sub-interval gradient and J_n at u0 for the full rotor problem, N=128 (sampled steps)."""
    w = W.config("rotor41")
    phi = O.intermediate_states(w, w.u0)
    g, Jn = O.subinterval_all(w, phi, w.u0)
    idx = np.arange(0, w.Nt, 13)
    return {"workload": "rotor41", "N": w.N, "grad_idx": idx.tolist(), "grad": g[idx].tolist(),
            "grad_l2": float(np.linalg.norm(g)), "Jn": Jn.tolist(),
            "phi_re_sample": phi[::8].real.tolist(), "phi_im_sample": phi[::8].imag.tolist()}


def gp512():
    """Full condensate benchmark problem: 512-point grid, Nt=10000, N=64, 20 iterations, rho=0.1
    (iterates of the nonlinear ISM with L = 1 do not depend on N either)."""
    w = W.gp_bec()
    t0 = time.time()
    u, J, F, E = G.ism_solve(w, w.u0, w.iters, w.rho)
    idx = np.arange(0, w.Nt, 37)
    g0 = G.global_gradient(w, w.u0)
    return {
        "workload": "gp512", "n": w.n, "Nt": w.Nt, "N": w.N, "iters": w.iters, "rho": w.rho,
        "source": "oracle.gp_oracle.ism_solve (FP64, numpy FFT split steps)",
        "J_hist": J.tolist(), "F_hist": F.tolist(), "err_hist": E.tolist(),
        "u_final_idx": idx.tolist(), "u_final": u[idx].tolist(),
        "grad0_idx": idx.tolist(), "grad0": g0[idx].tolist(), "grad0_l2": float(np.linalg.norm(g0)),
        "oracle_seconds": time.time() - t0,
    }


def ising1024_target():
    """The 10-spin chain of the benchmark with a seeded random unit target in place of |1^10>: from
    u0 ~ U[-0.1, 0.1] the overlap with |1^10> and its gradient are ~1e-10 and below, too small to
    compare FP32 propagation against, while a random target gives O(1) overlaps."""
    return W.with_random_target(W.config("ising1024"), 1103)


def ising1024():
    """Full 10-spin chain problem (random target, see ising1024_target): d=1024, Nt=50000, N=256,
    two iterations at rho=0.2, and the sub-interval gradient at u0 (sampled)."""
    w = ising1024_target()
    t0 = time.time()
    phi = O.intermediate_states(w, w.u0)
    g, Jn = O.subinterval_all(w, phi, w.u0)
    u, J, F, E = O.ism_solve(w, w.u0, 2, w.rho)
    idx = np.arange(0, w.Nt, 101)
    return {
        "workload": "ising1024", "d": w.d, "Nt": w.Nt, "N": w.N, "iters": 2, "rho": w.rho,
        "source": "oracle.ism_oracle (FP64, expm_multiply steps)",
        "J_hist": J.tolist(), "F_hist": F.tolist(), "err_hist": E.tolist(),
        "u_final_idx": idx.tolist(), "u_final": u[idx].tolist(),
        "grad_idx": idx.tolist(), "grad": g[idx].tolist(), "grad_l2": float(np.linalg.norm(g)), "Jn": Jn.tolist(),
        "oracle_seconds": time.time() - t0,
    }


JOBS = {"rotor41": rotor41, "rotor41_grad": rotor41_first_gradient, "gp512": gp512, "ising1024": ising1024}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for n in names:
        out = JOBS[n]()
        with open(os.path.join(HERE, f"{n}.json"), "w") as f:
            json.dump(out, f)
        print(n, "written")
