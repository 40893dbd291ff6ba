#!/usr/bin/env python
"""Benchmark of the ISM hot path on GB300.

A step is one pass of Algorithm 1 (propagator assembly, chain and intermediate states, sub-interval
forward/adjoint/gradient sweeps, control update) over a batch of independent rigid-rotor problems
(d = 41, Nt = 20000, N = 128, mixed precision, 4864 = 32 x 152 problems per launch by default).  The value is
ISM iterations per second summed over the batch; the line also carries the one-problem solve
latency (p50/p99 of complete 50-iteration solves), the plain FP64 one-problem path, the paper's
Crank-Nicolson scheme in FP64 (batched and one problem), a serving mix, the end-to-end rate through
host buffers, the roofline of the dominant kernel and the oracle on the host cores.
Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]
                    [--batch B] [--N N] [--Nt NT]
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # the oracle legs run single-threaded

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ISM gradient iters/s and complex state-steps/s vs plain FP64; p50/p99 solve latency"
UNIT = "ISM iterations/s"
DESCR = {"rotor41": "rigid rotor j<=40, maximise <cos theta>(T)",
         "spin16": "4 spins all-to-all ZZ, X control, |0000> -> |1111>",
         "ising1024": "10-spin open Ising chain, X control, |0^10> -> |1^10>",
         "gp512": "1D Gross-Pitaevskii condensate, 512-point grid, trap centre control, ground -> odd state",
         "gp512dw": "1D Gross-Pitaevskii condensate, 512-point grid, double-well splitting control, "
                    "harmonic ground state -> split-trap ground state",
         "spin5": "5 coupled spins, 10 controls (u_x, u_y per spin), density matrix in Liouville space, "
                  "I_x(1) -> I_x(5)",
         "dense256": "random dense real-symmetric H0, H1 (d = 256) on the tensor cores, random unit target"}
SAMPLE_DIV = {"dense256": 8, "rotor41": 8, "spin16": 1, "ising1024": 64, "gp512": 8, "gp512dw": 8, "spin5": 256}
# independent solves per launch: multiples of the 152 SMs (rotor41: two CTAs of 16 problems per SM in
# the wide lane layout of the direct sweeps; spin16: two CTAs of 8; one CTA per SM and direction for
# the CTA-wide kinds; two 152-CTA waves for the grid model)
BATCH_DEFAULT = {"dense256": 2432, "rotor41": 4864, "spin16": 2432, "ising1024": 152, "gp512": 1520, "gp512dw": 1520, "spin5": 152}
SOLVE_ITERS = {"dense256": 20, "rotor41": 50, "spin16": 20, "ising1024": 20, "gp512": 20, "gp512dw": 20, "spin5": 20}   # oracle sample = Nt/div steps, N/div sub-intervals
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_GB300 = 2070.0   # fallback when nvidia-smi cannot be read



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="rotor41")
    ap.add_argument("--N", type=int, default=None, help="sub-intervals (default: the workload's own)")
    ap.add_argument("--Nt", type=int, default=None,
                    help="time steps (default: the workload's own; smaller for profiler captures)")
    ap.add_argument("--batch", type=int, default=None, help="problems per launch (default: per workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cn", action="store_true", help="skip the Crank-Nicolson (Sec. 3 scheme) leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the full-size lines of the other configurations (spin16, gp512, ising1024)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


# ------------------------------------------------------------------------------ clocks sampling
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------ work accounting
def nnz_of(kind: str, d: int) -> int:
    if kind == "tridiag":
        return 3 * d - 2
    if kind == "bitflip":
        return d * (1 + int(round(np.log2(d))))
    if kind == "pauli":   # diagonal + an X and a Y flip per bit (the Y flips count as complex x real too)
        return d * (1 + 2 * int(round(np.log2(d))))
    return d * d


def cheb_flops(kind: str, d: int, y_apps: int, terms: int, substeps: int) -> float:
    """Algorithmic flops of the Chebyshev propagation: each application of the scaled Hamiltonian to
    a complex d-vector costs 4 nnz (complex x real multiply-adds) + 2d (recurrence subtraction), each
    accumulated term 4d, each exp sub-step's global phase 6d."""
    return float(y_apps) * (4 * nnz_of(kind, d) + 2 * d) + float(terms) * 4 * d + float(substeps) * 6 * d


KERNEL_SOURCES = ("ism_device.cuh", "ism_kernels.cuh", "ism_launch_impl.cuh", "ism_kern_tridiag.cu")


def kernel_source_hash(files=KERNEL_SOURCES) -> str:
    """Hash of the device code and launch configurations of the small-d Chebyshev kernels
    (k_cheb_prep, k_gsweep, k_subinterval, ...): a captured DRAM traffic is reported only while
    those kernels are the ones it was captured on."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1603_01237_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size launch divided by its
# problems, from a one-pass ncu capture of the default step (4864 rotor problems: k_gsweep in the wide
# lane layout); reported only while the kernel sources hash to the captured build.
TRAFFIC_PER_PROBLEM = {
    ("k_gsweep", "rotor41", "mixed"): {"bytes_per_problem": (1193538304 + 806773248) / 4864, "source_hash": "73cb90b7a0d46563"},
    ("k_subfwd", "rotor41", "mixed"): {"bytes_per_problem": (2211457792 + 2292974592) / 4864, "source_hash": "73cb90b7a0d46563"},
}


def traffic_of(kernel: str, workload: str, batch: int, precision: str):
    rec = TRAFFIC_PER_PROBLEM.get((kernel, workload, precision))
    if rec is None or rec["source_hash"] != kernel_source_hash():
        return None
    return rec["bytes_per_problem"] * batch


def measured_peaks() -> dict:
    """HBM copy bandwidth and bf16 GEMM rate measured on this GPU model, else the stated fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def gp_pair_flops(n: int) -> float:
    """Algorithmic flops of one split step of the grid model: an FFT pair (2 x 5 n log2 n) and two
    pointwise complex products (2 x 6n)."""
    return 10.0 * n * np.log2(n) + 12.0 * n


_PEAKS = {}


def alu_peak(P, which: str) -> dict:
    """The ALU roofline's peak: the FMA rate measured on this GPU by the library's own probe
    (ism_measure_peak: independent packed-FFMA2 or FP64 FMA chains on every SM, best of three timed
    launches), beside the figure derived from the device's SM count and the sampled maximum clock."""
    if which not in _PEAKS:
        import torch

        from paper_1603_01237_gb300 import abi

        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = max_sm_mhz()
        per = FP32_LANES_PER_SM * 2 if which == "fp32" else 2 * 2   # flops per SM per clock
        derived = sms * per * mhz * 1e6 / 1e12
        try:
            meas = abi.measure_peak(which)
            _PEAKS[which] = {"peak": meas, "source": f"measured: ism_measure_peak({which}) on {sms} SMs "
                                                     f"(derived {derived:.1f} from {sms} SMs x {per} flop/clk x {mhz:g} MHz)"}
        except Exception as exc:   # noqa: BLE001 - reported in the line
            _PEAKS[which] = {"peak": derived, "source": f"derived: {sms} SMs x {per} flop/clk x {mhz:g} MHz "
                                                        f"(measurement failed: {exc})"}
    return _PEAKS[which]


def max_sm_mhz() -> float:
    """The GPU's maximum SM clock as nvidia-smi reports it (clocks.max.sm), else the GB300 figure."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:   # noqa: BLE001
        return SM_MAX_MHZ_GB300


# ------------------------------------------------------------------------------ CPU oracle
_GP_STATES = {}


def load_workload(cfg: str, N=None, Nt=None):
    """The named synthetic workload (workloads/): the linear configurations or the 512-point grid."""
    import workloads as W

    if cfg == "gp512":
        w = W.gp_bec(Nt=Nt or 10000, N=N or 64, states=_GP_STATES.get("gp512"))
        _GP_STATES["gp512"] = (w.psi_i, w.psi_f)
        return w
    if cfg == "gp512dw":
        w = W.gp_double_well(Nt=Nt or 10000, N=N or 64, states=_GP_STATES.get("gp512dw"))
        _GP_STATES["gp512dw"] = (w.psi_i, w.psi_f)
        return w.with_(rho=0.05)
    if cfg == "spin5":
        return W.spin5_liouville(Nt=Nt or 32768, N=N or 128).with_(rho=100.0, iters=20)
    if cfg == "dense256":
        return W.random_dense(256, 401, T=(Nt or 1000) / 1000.0, Nt=Nt or 1000, N=N or 16, u_amp=0.5)
    return W.config(cfg, N=N, Nt=Nt)


def dim_of(w) -> int:
    return int(w.n) if getattr(w, "kind", "") == "gp" else int(w.d)


def oracle_sample(cfg: str, N_full: int):
    """One ISM iteration of the oracle on a time-truncated sample of the workload: Nt/div steps with
    N/div sub-intervals (same d and steps per sub-interval).  Returns (seconds, scale to full)."""
    from oracle import gp_oracle, ism_oracle

    full = load_workload(cfg, N=N_full)
    div = SAMPLE_DIV.get(cfg, 8)
    Nt_s = max(1, full.Nt // div)
    N_s = max(1, full.N // div)
    w = load_workload(cfg, N=N_s, Nt=Nt_s)
    from oracle import mc_oracle

    O = gp_oracle if cfg.startswith("gp512") else mc_oracle if cfg == "spin5" else ism_oracle
    t0 = time.perf_counter()
    O.ism_iteration(w, w.u0, w.rho, w.local_iters)
    dt = time.perf_counter() - t0
    return dt, Nt_s / full.Nt, f"one oracle ISM iteration on {cfg} truncated to Nt={Nt_s}, N={N_s} " \
                               f"(same d and steps per sub-interval), scaled by Nt_sample/Nt = {Nt_s / full.Nt:g}"


# ------------------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import workloads as W

    full = load_workload(args.config, N=args.N)
    times = []
    sample = ""
    scale = 1.0
    for s in range(args.warmup + args.steps):
        dt, scale, sample = oracle_sample(args.config, args.N)
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) * scale / tot * 1.0    # full-size ISM iterations per second
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        # ms_per_step is the measured wall time of one timed step (one sample iteration); value scales
        # the sample's rate to full-size iterations, so value != 1000 / ms_per_step here
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: {DESCR.get(args.config, args.config)} (d={dim_of(full)}), "
                               f"T={full.T:g}, Nt={full.Nt}, N={full.N}, one problem", "precision": "fp64 (oracle)",
                   "step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ multi-rank timing
def slowest_rank_ms(ms: float, world: int, device: str) -> float:
    """The job's time: the maximum over ranks of each rank's timed region (a no-op for one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(batch: int, steps: int, world: int, ms: float) -> float:
    """ISM iterations per second of the whole job: every rank solves its own batch (weak scaling)."""
    return batch * steps * world / (ms / 1e3)


# ------------------------------------------------------------------------------ serving mix
def serving_request(W, rng, k: int):
    """One request of the serving mix, as the packed C-ABI problem (no dense matrices): a spin system of
    d = 16 (4 spins, all-to-all ZZ), 64, 256 or 1024 (open chains of 6, 8, 10 sites), each with its own
    coupling draw J ~ U[0.5, 1.5], X control on every spin, |0..0> -> |1..1>, T = 10; or the rigid rotor
    of the rotor benchmark (d = 41, <cos theta> objective, T = pi).  Nt ~ U{1000..50000}, N from
    {8, 32, 128}, controls drawn like the benchmark's initial guesses, 20 iterations, mixed precision.
    Returns (name, problem arrays, u0, rho)."""
    kind = int(rng.integers(0, 5))
    Nt = int(rng.integers(1000, 50001))
    N = int(rng.choice([8, 32, 128]))
    if kind == 4:
        return "rotor41", W.config("rotor41", Nt=Nt, N=N), rng.uniform(-1.0, 1.0, Nt), 1.0
    q = (4, 6, 8, 10)[kind]
    d = 1 << q
    pairs = [(i, j) for i in range(q) for j in range(i + 1, q)] if q == 4 else [(i, i + 1) for i in range(q - 1)]
    J = np.random.default_rng(50000 + k).uniform(0.5, 1.5, size=len(pairs))
    prob = {"d": d, "Nt": Nt, "N": N, "T": 10.0, "H0": W._zz_diagonal(q, pairs, J), "H1": np.ones(q),
            "psi_i": np.eye(1, d, 0)[0].astype(np.complex128), "psi_f": np.eye(1, d, d - 1)[0].astype(np.complex128)}
    return ("spin16" if q == 4 else f"chain{d}"), prob, rng.uniform(-0.1, 0.1, Nt), 0.2


def serving_mix(P, W, seed: int, window_s: float = 10.0, rate: float = 200.0, slots: int = 16):
    """The serving workload: Poisson arrivals at `rate`/s for a time-bounded window of `window_s`
    seconds (the full workload is 10 000 requests at the same rate), continuous batching on the
    server (ism_server_*: shared plans per (kind, d, N, objective), rows refilled between ISM passes,
    HBM-budget admission).  Reports requests/s over the makespan, p50/p99 latency, how many requests a
    shared pass carried, and one-at-a-time FP64 (the library in FP64, one request per plan) estimated
    per request from timed FP64 iterations of each model (a full FP64 replay would take hours)."""
    import torch

    from paper_1603_01237_gb300 import abi

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, int(rate * window_s * 1.5) + 10)
    arrivals = np.cumsum(gaps)
    n_req = int(np.searchsorted(arrivals, window_s))
    reqs = [serving_request(W, rng, k) for k in range(n_req)]

    def packed(name, prob, u0, rho, precision="mixed"):
        """(ism_problem, ism_options, arrays to keep alive) of a request."""
        if name == "rotor41":
            return abi.problem_and_options(prob, precision=precision, rho=rho)
        keep = [np.ascontiguousarray(prob["H0"]), np.ascontiguousarray(prob["H1"]),
                prob["psi_i"].view(np.float64).copy(), prob["psi_f"].view(np.float64).copy()]
        pr = abi.IsmProblem(d=prob["d"], kind=abi.ISM_H_BITFLIP, H0=abi._ptr(keep[0]), H1=abi._ptr(keep[1]),
                            psi_i=abi._ptr(keep[2]), objective=abi.ISM_OBJ_OVERLAP, psi_f=abi._ptr(keep[3]), O=None,
                            T=prob["T"], Nt=prob["Nt"], N=prob["N"], alpha=None, batch=1, controls=1)
        op = abi.IsmOptions(precision=abi.ISM_MIXED if precision == "mixed" else abi.ISM_FP64, local_iters=1,
                            rho=float(rho), cheb_tol=0.0, max_spin_iters=0, subproblem_form=0, step1=0, scheme=0,
                            ckpt_stride=0)
        return pr, op, keep

    subs = [packed(*r) for r in reqs]
    with P.Server(slots=slots, hbm_budget_bytes=64 << 30) as srv:
        pr, op, keep = subs[0]
        srv.result(srv.submit_problem(pr, op, reqs[0][2], 1))   # warm-up: module load, first plan
        t0 = time.perf_counter()
        ids = []
        for (pr, op, keep), (name, prob, u0, rho), t_arr in zip(subs, reqs, arrivals[:n_req]):
            delay = t0 + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit_problem(pr, op, u0, 20))
        lat = [srv.result(i)[2][2] for i in ids]
        makespan = time.perf_counter() - t0
        st = srv.stats()
    # one-at-a-time FP64: seconds per step of one FP64 ISM iteration of each model (one problem per plan)
    per_step = {}
    for name, prob, u0, rho in reqs:
        if name in per_step:
            continue
        if name == "rotor41":
            ps = W.config("rotor41", Nt=2000, N=32)
        else:
            ps = dict(prob, Nt=2000, N=32)
        pr, op, keep = packed(name, ps, u0[:2000], rho, precision="fp64")
        plan = abi.Plan.from_problem(pr, op, keep)
        uu = np.ascontiguousarray(u0[:2000][None, :])
        J = np.empty((1, 3))
        plan.ism_iterate(1, uu, None, None)
        t1 = time.perf_counter()
        plan.ism_iterate(2, uu, J, None)
        per_step[name] = (time.perf_counter() - t1) / 3 / 2000   # 2 iterations and the final evaluation
        plan.close()
    est = sum(21 * per_step[name] * (prob.Nt if name == "rotor41" else prob["Nt"]) for name, prob, u0, rho in reqs)
    return {"requests": n_req, "arrival_rate_per_s": rate, "arrival_window_s": window_s, "slots": slots,
            "iterations": 20, "requests_per_s": n_req / makespan, "makespan_s": makespan,
            "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
            "shared_passes": st["passes"], "requests_per_shared_pass": st["request_passes"] / max(1, st["passes"]),
            "max_requests_in_a_pass": st["max_rows"], "shared_plans": st["groups"], "own_plans": st["single"],
            "one_at_a_time_fp64_requests_per_s": n_req / est,
            "one_at_a_time_fp64": "estimated: 21 x Nt x (seconds per step of a timed 2000-step FP64 ISM iteration of "
                                  "the request's model, one problem per plan), summed over the requests",
            "mix": "d in {16 (4 spins all-to-all), 64, 256, 1024 (open chains of 6, 8, 10 sites)} with per-request "
                   "coupling draws, and the rigid rotor (d = 41); Nt ~ U{1000..50000}, N in {8, 32, 128}, 20 "
                   "iterations, mixed precision; Poisson arrivals, time-bounded window"}


# ------------------------------------------------------------------------------ our arm
# ------------------------------------------------------------------------------ Crank-Nicolson leg
CN_BATCH = 1024   # saturates the FP64 pipe (256 problems per launch take the same time per launch)


def cn_jacobi_iterations(w, tol: float = 1e-17) -> int:
    """Jacobi iterations per Crank-Nicolson solve, as the parameter kernel chooses them:
    rho = (tau/2)(off0 + max|u| off1), rho^K <= tol."""
    off = lambda A: float(np.max(np.abs(A - np.diag(np.diag(A))).sum(axis=1)))
    rho = 0.5 * w.T / w.Nt * (off(w.H0) + float(np.max(np.abs(w.u0))) * off(w.H1)) * (1 + 1e-6)
    return 1 if rho <= 0 else max(1, int(np.ceil(np.log(tol) / np.log(rho))))


def cn_flops_per_state_step(d: int, K: int) -> float:
    """FP64 flops of one Crank-Nicolson step of one state with tridiagonal H (per complex element:
    H v 12, right-hand side 4, first Jacobi iteration 6, each further one 16 -- off-diagonal part
    of H 6, update 4, diagonal inverse 6)."""
    return d * (22.0 + 16.0 * (K - 1))


def crank_nicolson_leg(P, w, stream, steps: int, cpu: bool):
    """The Sec. 3 scheme in FP64 on the same rotor problem: batched direct sweeps (CN_BATCH problems
    per launch; inputs larger than L2), one-problem latency by the assembly path, the FP64 ALU
    roofline of the dominant kernel and the Crank-Nicolson oracle on a bounded sample."""
    import torch

    K = cn_jacobi_iterations(w)
    B = CN_BATCH
    rng = np.random.default_rng(4000)
    amp = float(np.max(np.abs(w.u0)))
    U0 = np.stack([w.u0] + [rng.uniform(-amp, amp, w.Nt) for _ in range(B - 1)])
    plan = P.Plan(w, precision="fp64", batch=B, stream=stream, scheme="crank_nicolson", step1=2)
    u = torch.tensor(U0, dtype=torch.float64, device="cuda").contiguous()
    plan.ism_iterate(1, u, None, None)
    n = max(2, steps // 10)
    plan.ism_set_profiling(True)
    plan.ism_get_stats(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        plan.ism_iterate(n, u, None, None)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    st = plan.ism_get_stats(reset=True)
    plan.close()
    names = ["k_gsweep", "k_phi", "k_subfwd"]
    dom = 0 if st["ms"][0] >= st["ms"][2] else 2
    ms_launch = st["ms"][dom] / n
    flops = 2.0 * w.Nt * B * cn_flops_per_state_step(int(w.d), K)   # two sweeps per launch
    achieved = flops / (ms_launch / 1e3) / 1e12
    pk = alu_peak(P, "fp64")
    roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": pk["peak"],
            "unit": "TFLOP/s", "frac": achieved / pk["peak"], "traffic": None, "peak_source": pk["source"],
            "flops_per_launch": flops, "ms_per_launch": ms_launch}
    p1 = P.Plan(w, precision="fp64", batch=1, stream=stream, scheme="crank_nicolson")
    u1 = torch.tensor(w.u0, dtype=torch.float64, device="cuda").reshape(1, -1).contiguous()
    p1.ism_iterate(1, u1, None, None)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        p1.ism_iterate(3, u1, None, None)
        e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / 3
    p1.close()
    out = {"value": B / (ms / 1e3), "unit": UNIT, "batch": B, "ms_per_iteration": ms, "jacobi_iterations": K,
           "precision": "fp64", "l2": "inputs larger than L2 (trajectory slots 15.8 GB)",
           "latency_ms_per_iteration_batch1": ms1, "phase_share": {nm: st["ms"][i] / max(1e-12, sum(st["ms"]))
                                                                  for i, nm in enumerate(names)},
           "roofline": roof}
    # the FP32 Cayley step (mixed precision, hi + lo diagonal coefficients)
    Bm = 4864
    Um = np.stack([w.u0] + [rng.uniform(-amp, amp, w.Nt) for _ in range(Bm - 1)])
    pm = P.Plan(w, precision="mixed", batch=Bm, stream=stream, scheme="crank_nicolson")
    um = torch.tensor(Um, dtype=torch.float64, device="cuda").contiguous()
    pm.ism_iterate(1, um, None, None)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        pm.ism_iterate(n, um, None, None)
        e1.record(stream)
    torch.cuda.synchronize()
    msm = e0.elapsed_time(e1) / n
    pm.close()
    out["mixed"] = {"value": Bm / (msm / 1e3), "unit": UNIT, "batch": Bm, "ms_per_iteration": msm,
                    "accuracy": "J within 1e-5 and the gradient within 1e-4 relative of the FP64 "
                                "Crank-Nicolson oracle at this size (tested)"}
    if cpu:
        from oracle import cn_oracle

        div = SAMPLE_DIV.get("rotor41", 8)
        ws = W_config(w, Nt=w.Nt // div, N=max(1, w.N // div))
        tot, n_s = 0.0, 0
        while tot < 10.0 and n_s < 20:
            t0 = time.perf_counter()
            cn_oracle.ism_iteration(ws, ws.u0, ws.rho, ws.local_iters)
            tot += time.perf_counter() - t0
            n_s += 1
        out["cpu_baseline"] = {"value": n_s * (ws.Nt / w.Nt) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"one Crank-Nicolson oracle ISM iteration on rotor41 truncated to "
                                         f"Nt={ws.Nt}, N={ws.N}, scaled by {ws.Nt / w.Nt:g}; {n_s} repetitions, "
                                         f"{tot:.1f} s"}
    return out


def tf32_peak() -> dict:
    """The TF32 tensor rate: the measured bf16 GEMM rate (MEASURED_PEAKS.json, else the stated fallback)
    scaled by the nominal TF32/bf16 ratio (1.1 / 2.25 PFLOP/s dense)."""
    pk = measured_peaks()
    return {"peak": pk["bf16_tflops"] * 1.1 / 2.25,
            "source": f"{pk['source']} bf16 {pk['bf16_tflops']:g} TFLOP/s x 1.1/2.25 (nominal TF32/bf16 ratio)"}


def timed_iterations(P, w, B, stream, steps: int, warmup: int = 2, **kw):
    """ms per batched ISM iteration (CUDA events, mixed precision) and the plan's work/time accounting."""
    import torch

    rng = np.random.default_rng(7000)
    amp = float(np.max(np.abs(w.u0)))
    U0 = np.stack([w.u0] + [rng.uniform(-amp, amp, w.Nt) for _ in range(B - 1)])
    plan = P.Plan(w, precision="mixed", batch=B, stream=stream, **kw)
    u = torch.tensor(U0, dtype=torch.float64, device="cuda").contiguous()
    for _ in range(warmup):
        plan.ism_iterate(1, u, None, None)
    plan.ism_set_profiling(True)
    plan.ism_get_stats(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        plan.ism_iterate(steps, u, None, None)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = plan.ism_get_stats(reset=True)
    tc = plan.info(10) == 1
    plan.close()
    return ms, st, tc


def tensor_core_leg(P, W, stream, steps: int) -> dict:
    """Dense Hamiltonians on the tensor cores (d = 256; tcgen05, TF32 x 3 split operands): a genuinely
    dense random H, and the 8-spin chain (d = 256, 9 couplings per row) both as a dense matrix on the
    tensor cores and through the structured bit-flip path.  Executed tensor flops count every state's
    Y applications as 2 columns x 2 GEMM halves (H0, H1) x 3 split passes x 2 d^2 flops; useful flops
    are the algorithmic ones of the operator (dense: 4 d^2 + 2d per Y application of a complex state)."""
    d, B, Nt, N = 256, 2432, 1000, 16
    pk = tf32_peak()
    out = {"d": d, "batch": B, "Nt": Nt, "N": N, "peak_tf32": pk}
    dense = W.random_dense(d, 401, T=1.0, Nt=Nt, N=N, u_amp=0.5)
    ms, st, tc = timed_iterations(P, dense, B, stream, steps)
    tc_ms = st["ms"][0] + st["ms"][2]
    y = st["y_apps"][0] + st["y_apps"][1]
    executed = y * 24.0 * d * d
    useful = cheb_flops("dense", d, y, st["terms"][0] + st["terms"][1], st["substeps"][0] + st["substeps"][1])
    out["random_dense"] = {"tensor_cores": tc, "value": B / (ms / 1e3), "unit": UNIT, "ms_per_iteration": ms,
                           "tensor_tflops": executed / (tc_ms / 1e3) / 1e12,
                           "tensor_frac": executed / (tc_ms / 1e3) / 1e12 / pk["peak"],
                           "useful_tflops": useful / (tc_ms / 1e3) / 1e12,
                           "phase_share": {n: st["ms"][i] / max(1e-12, sum(st["ms"]))
                                           for i, n in enumerate(["k_tc_sweep (global)", "k_phi", "k_tc_sweep + k_tc_zgrad (sub)"])}}
    chain = W.with_random_target(W.spin_chain(8, 402, T=1.0, Nt=Nt, N=N), 403)
    ms_d, st_d, tc_d = timed_iterations(P, chain.with_(kind="dense"), B, stream, steps)
    ms_s, st_s, _ = timed_iterations(P, chain, B, stream, steps)
    y_s = st_s["y_apps"][0] + st_s["y_apps"][1]
    useful_s = cheb_flops("bitflip", d, y_s, st_s["terms"][0] + st_s["terms"][1], st_s["substeps"][0] + st_s["substeps"][1])
    out["spin_chain_8"] = {"dense_on_tensor_cores": {"value": B / (ms_d / 1e3), "ms_per_iteration": ms_d, "tensor_cores": tc_d},
                           "structured_bitflip": {"value": B / (ms_s / 1e3), "ms_per_iteration": ms_s,
                                                  "useful_tflops": useful_s / (ms_s / 1e3) / 1e12},
                           "structured_over_dense": ms_d / ms_s}
    return out


def W_config(w, Nt: int, N: int):
    """The same named workload at another Nt, N (same seed: u0 drawn at the new length)."""
    import workloads as W

    return W.config(w.name, Nt=Nt, N=N)


# precision each configuration is specified in, and the parity bar its full-size run is tested at
CONFIG_PRECISION = {"dense256": "mixed", "rotor41": "mixed", "spin16": "fp64", "gp512": "mixed", "gp512dw": "mixed", "ising1024": "mixed",
                    "spin5": "mixed"}
TESTED = {
    "rotor41": "J within 1e-5, controls within 1e-4, Err within 1e-4 of the FP64 oracle over 50 iterations, "
               "this 4864-problem plan included (tests/test_gpu_fullsize.py)",
    "spin16": "J, F and controls within 1e-9 of the FP64 oracle over 20 iterations (tests/test_gpu_parity.py)",
    "gp512": "J within 1e-5, controls within 1e-4 of the FP64 oracle over 20 iterations; gradient within 1e-4 "
             "(tests/test_gpu_fullsize.py)",
    "gp512dw": "J within 1e-5 over 2 iterations, gradient within 1e-4 (tests/test_gpu_gp.py)",
    "ising1024": "J within 1e-5, controls within 1e-4 of the FP64 oracle over 2 iterations; sub-interval gradient "
                 "within 1e-4 (tests/test_gpu_fullsize.py)",
    "spin5": "J within 1e-4 of the density-matrix oracle at the paper's size (tests/test_gpu_pauli.py)",
    "dense256": "states within 2e-5, gradient within 1e-4 relative and J within 1e-5 of the FP64 oracle on random "
                "dense d = 128 and 256 (tests/test_gpu_tc.py)",
}
SUB_CONFIGS = ("spin16", "gp512", "ising1024")


def state_steps_per_iteration(plan, w) -> tuple:
    """Complex state-steps (one U_j applied to one state) of one ISM iteration of one problem, as the
    plan's kernels execute them: 2 Nt for the global sweeps (direct) and, per sub-interval, psi and chi
    carried forward (2 Nt; the first local step of the two-trajectory form) or the literal
    sub-problem's forward sweep, its recomputation from the checkpoints and the adjoint (~3 Nt); the
    grid model's first local step takes the sub-problems' forward trajectories from the global forward
    sweep's stored states and runs their adjoints (2 Nt global + Nt sub-interval)."""
    if plan.gp:
        return 3 * w.Nt, "2 Nt global sweeps + Nt sub-interval adjoint steps (the sub-problems' forward trajectories are the global sweep's stored states)"
    return 4 * w.Nt, "2 Nt global sweeps + 2 Nt sub-interval sweeps (psi and chi forward)"


def oracle_worker(cfg: str, N, seconds: float):
    """One host process: repeat the bounded oracle sample for about `seconds`; (samples, busy s, scale)."""
    tot, n, scale, sample = 0.0, 0, 1.0, ""
    while tot < seconds and n < 50:
        dt, scale, sample = oracle_sample(cfg, N)
        tot += dt
        n += 1
    return n, tot, scale, sample


def cpu_baseline_of(cfg: str, N, seconds: float = 10.0) -> dict:
    """The oracle on the host: one process (the sequential t(eps, 1) of Sec. 4), and one process per host
    core running independent samples at once (the N-processor analogue); value = the all-core rate."""
    import concurrent.futures as cf
    import multiprocessing as mp

    n1, t1, scale, sample = oracle_worker(cfg, N, seconds)
    one = n1 * scale / t1
    cores = os.cpu_count() or 1
    allc, used = one, 1
    if cores > 1:
        try:   # spawn: this process has a CUDA context, a forked child would inherit it
            with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
                res = list(ex.map(oracle_worker, [cfg] * cores, [N] * cores, [seconds] * cores))
            allc = sum(n * sc / t for n, t, sc, _ in res)
            used = cores
        except Exception:   # noqa: BLE001 - the single-core figure stands
            pass
    return {"value": allc, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{sample}; {used} host processes at once, about {seconds:g} s each (the rate is summed over "
                      f"them)", "single_core": {"value": one, "cores": 1, "seconds": t1, "repetitions": n1},
            "host_cores": cores}


def measure_config(P, W, cfg: str, args, stream, steps: int, warmup: int, world: int, rank: int, N=None, Nt=None,
                   batch=None) -> dict:
    """Batched ISM iterations of one configuration at full size: CUDA-event time per iteration (L2
    flushed between steps), the roofline of the dominant phase (algorithmic flops from the kernels' work
    counters over the measured FMA peak) and the phase shares."""
    import torch

    w = load_workload(cfg, N=N, Nt=Nt)
    d = dim_of(w)
    B = batch or BATCH_DEFAULT.get(cfg, 1)
    prec = CONFIG_PRECISION.get(cfg, "mixed")
    plan = P.Plan(w, precision=prec, batch=B, stream=stream)
    rng = np.random.default_rng(2000 + rank)
    amp = float(np.max(np.abs(w.u0)))   # further problems: controls of the same amplitude as u0
    U0 = np.stack([w.u0] + [rng.uniform(-amp, amp, w.u0.shape) for _ in range(B - 1)])
    u_dev = torch.tensor(U0, dtype=torch.float64, device="cuda").contiguous()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2
    for _ in range(warmup):
        plan.ism_iterate(1, u_dev, None, None)
    plan.ism_set_profiling(True)
    plan.ism_get_stats(reset=True)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()                       # evict the previous step's working set from L2
            ev[k][0].record(stream)
            plan.ism_iterate(1, u_dev, None, None)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = slowest_rank_ms(sum(step_ms), world, "cuda")
    st = plan.ism_get_stats(reset=True)
    plan.ism_set_profiling(False)
    value = job_throughput(B, steps, world, tot_ms)
    ss, ss_how = state_steps_per_iteration(plan, w)

    large = plan.ks_large
    direct = plan.info(6) == 2   # Algorithm 1 (a)-(b) by direct sweeps
    sub = "k_subfwd"   # first local steps run the two-trajectory form in both precisions
    tc = plan.info(10) == 1
    if tc:
        names = ["k_tc_sweep (global)", "k_phi", "k_tc_sweep (sub)"]
        kernels = ["k_cheb_prep + k_tc_sweep", "k_phi", "k_tc_sweep + k_tc_zgrad"]
    elif plan.gp:
        names = ["k_gp_forward", "k_gp_adjoint", "k_gp_sub"]
        kernels = names
    elif plan.kind == "pauli":
        names = ["k_pauli_sweep", "k_phi", "k_pauli_sub"]
        kernels = ["k_pauli_prep + k_pauli_sweep", "k_phi", "k_pauli_sub"]
    elif large:
        names = ["k_lsweep", "k_phi", "k_lsub"]
        kernels = ["k_cheb_prep + k_lsweep", "k_phi", "k_lsub"]
    elif direct:
        names = ["k_gsweep", "k_phi", sub]
        kernels = ["k_cheb_prep + k_gsweep", "k_phi", sub]
    else:
        names = ["k_assemble", "k_chain", "k_sweeps2"]
        kernels = ["k_cheb_prep + k_assemble", "k_chain + k_phi", "k_sweeps2 + k_gradpass"]
    dom = int(np.argmax(st["ms"]))
    ms_launch = st["ms"][dom] / steps
    peaks = measured_peaks()
    if tc and dom in (0, 2):   # executed tensor flops: 2 columns x [H0; H1] x 3 split passes per Y application
        k = 0 if dom == 0 else 1
        flops = st["y_apps"][k] * 24.0 * d * d / steps
        achieved = flops / (ms_launch / 1e3) / 1e12
        pk = tf32_peak()
        roof = {"kernel": names[dom], "kernels_timed": kernels[dom], "bound": "tensor", "achieved": achieved,
                "peak": pk["peak"], "unit": "TFLOP/s", "frac": achieved / pk["peak"], "traffic": None,
                "peak_source": pk["source"], "flops_per_launch": flops, "ms_per_launch": ms_launch,
                "useful_tflops": cheb_flops("dense", d, st["y_apps"][k], st["terms"][k], st["substeps"][k]) / steps
                / (ms_launch / 1e3) / 1e12}
    elif plan.gp or dom in (0, 2) or large or direct:
        if plan.gp:   # FFT pairs counted by the kernels: forward, adjoint, sub-interval
            pairs = [st["y_apps"][0], st["terms"][0], st["terms"][1]][dom]
            flops = pairs * gp_pair_flops(d) / steps
        elif dom == 1:   # k_phi
            flops = 8.0 * B * (w.N + 1) * d
        else:
            k = 0 if dom == 0 else 1
            flops = cheb_flops(plan.kind, d, st["y_apps"][k], st["terms"][k], st["substeps"][k]) / steps
        achieved = flops / (ms_launch / 1e3) / 1e12
        pk = alu_peak(P, "fp64" if prec == "fp64" else "fp32")
        roof = {"kernel": names[dom], "kernels_timed": kernels[dom], "bound": "alu", "achieved": achieved,
                "peak": pk["peak"], "unit": "TFLOP/s", "frac": achieved / pk["peak"],
                "traffic": traffic_of(names[dom], cfg, B, prec), "peak_source": pk["source"], "flops_per_launch": flops,
                "ms_per_launch": ms_launch}
    else:
        # algorithmic bytes: every stored propagator tile read once per chain, both staged state chains written
        tile = plan.info(4)
        nbytes = B * (2 * w.N * tile + 2 * (w.N + 1) * d * 8)
        achieved = nbytes / (ms_launch / 1e3) / 1e9
        roof = {"kernel": names[dom], "kernels_timed": kernels[dom], "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic_of(names[dom], cfg, B, prec), "peak_source": peaks["source"], "bytes_per_launch": nbytes,
                "ms_per_launch": ms_launch}
    return {"plan": plan, "w": w, "U0": U0, "B": B, "d": d, "prec": prec, "value": value, "steps": steps,
            "ms_per_step": tot_ms / steps, "step_ms": step_ms, "state_steps": ss, "state_steps_how": ss_how,
            "roofline": roof, "phase_share": {n: st["ms"][i] / max(1e-12, sum(st["ms"])) for i, n in enumerate(names)},
            "gpu_launches": int(st["kernels"]), "clocks": clk}


def config_summary(cfg: str, m: dict, cpu) -> dict:
    w = m["w"]
    return {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"], "steps": m["steps"],
            "workload": f"{cfg}: {DESCR.get(cfg, cfg)} (d={m['d']}), T={w.T:g}, Nt={w.Nt}, N={w.N}, "
                        f"batch={m['B']} per GPU", "precision": m["prec"],
            "state_steps_per_s": m["value"] * m["state_steps"], "state_steps_per_iteration": m["state_steps_how"],
            "roofline": m["roofline"], "phase_share": m["phase_share"], "cpu_baseline": cpu,
            "tested": TESTED.get(cfg), "clocks": m["clocks"]}


def run_ours(args):
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P
    import workloads as W

    stream = torch.cuda.Stream()
    m = measure_config(P, W, args.config, args, stream, args.steps, args.warmup, world, rank, N=args.N, Nt=args.Nt,
                       batch=args.batch)
    plan, w, U0, B, d = m["plan"], m["w"], m["U0"], m["B"], m["d"]

    # e2e through the C ABI with host buffers: H2D of u, one iteration, D2H of u and Err
    u_host = torch.tensor(U0, dtype=torch.float64).pin_memory()
    err_host = torch.empty((B, 1), dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.ism_iterate(1, u_host, None, err_host)
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        plan.ism_iterate(1, u_host, None, err_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": B / statistics.mean(e2e_t) * world, "unit": UNIT,
           "h2d_bytes_per_step": int(u_host.numel() * 8),
           "d2h_bytes_per_step": int(u_host.numel() * 8 + err_host.numel() * 8)}
    plan.close()

    # plain FP64, one problem per launch
    fp64 = None
    if not args.no_fp64:
        p64 = P.Plan(w, precision="fp64", batch=1, stream=stream)
        u64 = torch.tensor(w.u0, dtype=torch.float64, device="cuda").reshape(1, -1).contiguous()
        p64.ism_iterate(1, u64, None, None)
        n64 = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            p64.ism_iterate(n64, u64, None, None)
            e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        fp64 = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_iteration": ms64, "batch": 1}
        p64.close()

    # solve latency: complete solves (the workload's iteration count) of one problem per launch
    it_solve = SOLVE_ITERS.get(args.config, 20)
    p1 = P.Plan(w, precision=m["prec"], batch=1, stream=stream)
    u1 = torch.tensor(w.u0, dtype=torch.float64, device="cuda").reshape(1, -1).contiguous()
    u1_0 = u1.clone()
    p1.ism_iterate(it_solve, u1, None, None)
    n_solves = 10 if d <= 64 else 2
    sol_ms = []
    with torch.cuda.stream(stream):
        for _ in range(n_solves):
            u1.copy_(u1_0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p1.ism_iterate(it_solve, u1, None, None)
            e1.record(stream)
            e1.synchronize()
            sol_ms.append(e0.elapsed_time(e1))
    p1.close()
    solve = {"batch": 1, "iterations": it_solve, "solves": n_solves, "p50_ms": float(np.percentile(sol_ms, 50)),
             "p99_ms": float(np.percentile(sol_ms, 99)), "ms_per_iteration": float(np.median(sol_ms)) / it_solve}

    serving = None if args.no_serving else serving_mix(P, W, seed=3000 + rank)
    cn = None
    if not args.no_cn and getattr(w, "kind", "") == "tridiag":
        cn = crank_nicolson_leg(P, w, stream, args.steps, cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))

    tcleg = None
    if args.config == "rotor41" and not args.no_configs and args.N is None and args.Nt is None:
        tcleg = tensor_core_leg(P, W, stream, 3)

    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    cpu = cpu_baseline_of(args.config, args.N) if want_cpu else None

    # the other configurations at full size, in their own precision, fewer timed steps
    others = {}
    if args.config == "rotor41" and not args.no_configs and args.N is None and args.Nt is None:
        for cfg in SUB_CONFIGS:
            mc = measure_config(P, W, cfg, args, stream, max(3, min(args.steps, 5)), 3, world, rank)
            mc["plan"].close()
            others[cfg] = config_summary(cfg, mc, cpu_baseline_of(cfg, None, 5.0) if want_cpu else None)

    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 propagation, f64 states/overlaps/update" if m["prec"] == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.config}: {DESCR.get(args.config, args.config)} (d={d}), T={w.T:g}, "
                               f"Nt={w.Nt}, N={w.N}, batch={B} per GPU", "d": d, "Nt": w.Nt, "N": w.N, "batch": B,
                   "precision": m["prec"], "l2": "flushed between steps (512 MB write, outside the timed events)"},
        "state_steps_per_s": m["value"] * m["state_steps"], "state_steps_per_iteration": m["state_steps_how"],
        "step_ms_p50": statistics.median(m["step_ms"]), "step_ms_p99": float(np.percentile(m["step_ms"], 99)),
        "tested": TESTED.get(args.config),
        "solve_latency": solve,
        "serving": serving,
        "fp64_plain": fp64,
        "crank_nicolson": cn,
        "configs": others or None,
        "tensor_cores": tcleg,
        "phase_share": m["phase_share"],
        "roofline": m["roofline"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": m["gpu_launches"],
        "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
