"""Write the stored expected values used by the full-size GPU parity tests.

Every number here comes from the FP64 oracle (oracle/ism_oracle.py) run on the seeded workloads of
the `workloads` package; nothing is read from the CUDA path.

    python tests/golden/make_golden.py rotor41      # ~15-30 min on one core
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


JOBS = {"rotor41": rotor41, "rotor41_grad": rotor41_first_gradient}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for n in names:
        out = JOBS[n]()
        with open(os.path.join(HERE, f"{n}.json"), "w") as f:
            json.dump(out, f)
        print(n, "written")
