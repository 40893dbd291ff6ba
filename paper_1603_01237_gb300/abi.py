"""ctypes binding of libism.so (include/ism.h): the same entry points, argument marshalling only.

Array arguments may be numpy float64 arrays (host) or torch tensors (host or CUDA); every step of
the computation runs in the library's CUDA kernels.  There is no CPU fallback: if libism.so is
missing or fails to load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB = None
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libism.so")

ISM_OK, ISM_EINVAL, ISM_ENOMEM, ISM_ECUDA, ISM_ENONFINITE, ISM_ETIMEOUT, ISM_EUNSUPPORTED = range(7)
ISM_FP64, ISM_MIXED = 0, 1
ISM_H_DENSE, ISM_H_BITFLIP, ISM_H_TRIDIAG, ISM_H_GRID_GP, ISM_H_GRID_GP_DOUBLE_WELL, ISM_H_PAULI = 0, 1, 2, 3, 4, 5
ISM_OBJ_OVERLAP, ISM_OBJ_OBSERVABLE = 0, 1
ISM_SCHEME_CHEBYSHEV, ISM_SCHEME_CRANK_NICOLSON = 0, 1
_SCHEME = {"chebyshev": ISM_SCHEME_CHEBYSHEV, "crank_nicolson": ISM_SCHEME_CRANK_NICOLSON}

STATUS_NAMES = {0: "ISM_OK", 1: "ISM_EINVAL", 2: "ISM_ENOMEM", 3: "ISM_ECUDA", 4: "ISM_ENONFINITE",
                5: "ISM_ETIMEOUT", 6: "ISM_EUNSUPPORTED"}

EXPORTS = ("ism_plan", "ism_plan_destroy", "ism_intermediate_states", "ism_subinterval_grad",
           "ism_iterate", "ism_evaluate", "ism_gradient", "ism_set_profiling", "ism_get_stats", "ism_plan_info",
           "ism_plan_footprint", "ism_server_create", "ism_server_submit", "ism_server_poll",
           "ism_server_release", "ism_server_stats", "ism_server_destroy",
           "ism_subinterval_grad_noalloc", "ism_measure_peak", "ism_last_error", "ism_version")


class IsmProblem(C.Structure):
    _fields_ = [("d", C.c_int), ("kind", C.c_int), ("H0", C.c_void_p), ("H1", C.c_void_p),
                ("psi_i", C.c_void_p), ("objective", C.c_int), ("psi_f", C.c_void_p), ("O", C.c_void_p),
                ("T", C.c_double), ("Nt", C.c_int), ("N", C.c_int), ("alpha", C.c_void_p), ("batch", C.c_int),
                ("controls", C.c_int), ("H0_imag", C.c_void_p), ("H1_imag", C.c_void_p)]


class IsmOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("local_iters", C.c_int), ("rho", C.c_double),
                ("cheb_tol", C.c_double), ("max_spin_iters", C.c_int), ("subproblem_form", C.c_int),
                ("step1", C.c_int), ("scheme", C.c_int), ("ckpt_stride", C.c_int)]


class IsmStats(C.Structure):
    _fields_ = [("ms", C.c_double * 3), ("launches", C.c_longlong * 3), ("y_apps", C.c_ulonglong * 2),
                ("terms", C.c_ulonglong * 2), ("substeps", C.c_ulonglong * 2), ("kernels", C.c_longlong),
                ("norm_drift", C.c_double)]


class IsmServerOptions(C.Structure):
    _fields_ = [("slots", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("group_capacity", C.c_int),
                ("group_max_steps", C.c_int)]


ISM_REQ_QUEUED, ISM_REQ_RUNNING, ISM_REQ_DONE, ISM_REQ_FAILED = 0, 1, 2, 3


class IsmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str | None = None):
    """Load libism.so (once).  Raises OSError if it is missing: build it with
    ``paper_1603_01237_gb300.build.build()``."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libism.so not found at {p}; run paper_1603_01237_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.ism_plan.argtypes = [C.POINTER(IsmProblem), C.POINTER(IsmOptions), vp, C.POINTER(vp)]
    lib.ism_plan.restype = i
    lib.ism_plan_destroy.argtypes = [vp]
    lib.ism_plan_destroy.restype = i
    lib.ism_intermediate_states.argtypes = [vp, vp, vp]
    lib.ism_intermediate_states.restype = i
    lib.ism_subinterval_grad.argtypes = [vp, vp, vp, vp, vp]
    lib.ism_subinterval_grad.restype = i
    lib.ism_iterate.argtypes = [vp, i, vp, vp, vp]
    lib.ism_iterate.restype = i
    lib.ism_evaluate.argtypes = [vp, vp, vp, vp]
    lib.ism_evaluate.restype = i
    lib.ism_gradient.argtypes = [vp, vp, vp, vp]
    lib.ism_gradient.restype = i
    lib.ism_set_profiling.argtypes = [vp, i]
    lib.ism_set_profiling.restype = i
    lib.ism_get_stats.argtypes = [vp, C.POINTER(IsmStats), i]
    lib.ism_get_stats.restype = i
    lib.ism_plan_info.argtypes = [vp, i]
    lib.ism_plan_info.restype = C.c_longlong
    lib.ism_plan_footprint.argtypes = [C.POINTER(IsmProblem), C.POINTER(IsmOptions), C.POINTER(C.c_size_t)]
    lib.ism_plan_footprint.restype = i
    lib.ism_server_create.argtypes = [C.POINTER(IsmServerOptions), C.POINTER(vp)]
    lib.ism_server_create.restype = i
    lib.ism_server_submit.argtypes = [vp, C.POINTER(IsmProblem), C.POINTER(IsmOptions), vp, i,
                                      C.POINTER(C.c_longlong)]
    lib.ism_server_submit.restype = i
    lib.ism_server_poll.argtypes = [vp, C.c_longlong, i, C.POINTER(i), vp, vp, vp]
    lib.ism_server_poll.restype = i
    lib.ism_server_release.argtypes = [vp, C.c_longlong]
    lib.ism_server_release.restype = i
    lib.ism_server_stats.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.ism_server_stats.restype = i
    lib.ism_server_destroy.argtypes = [vp]
    lib.ism_server_destroy.restype = i
    lib.ism_subinterval_grad_noalloc.argtypes = [C.POINTER(IsmProblem), i, vp, vp, vp, vp, vp]
    lib.ism_subinterval_grad_noalloc.restype = i
    lib.ism_measure_peak.argtypes = [i, C.POINTER(d)]
    lib.ism_measure_peak.restype = i
    lib.ism_last_error.argtypes = []
    lib.ism_last_error.restype = C.c_char_p
    lib.ism_version.argtypes = []
    lib.ism_version.restype = C.c_char_p
    _LIB = lib
    return lib


def _check(rc: int):
    if rc != ISM_OK:
        msg = load().ism_last_error().decode(errors="replace")
        raise IsmError(rc, msg)


_ARRAY_DTYPES = ("float64", "complex128")   # every array of the C ABI is double (complex: interleaved pairs)


def _ptr(x):
    """Address of a numpy array / torch tensor (host or device), or None.  Only float64 and complex128
    data are accepted: the library reads every array as doubles, so a narrower type would be read past
    its end."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        if x.dtype.name not in _ARRAY_DTYPES:
            raise TypeError(f"arrays must be float64 or complex128, not {x.dtype.name}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if str(x.dtype).replace("torch.", "") not in _ARRAY_DTYPES:
            raise TypeError(f"tensors must be float64 or complex128, not {x.dtype}")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _doubles(x) -> int:
    """Number of doubles an array or tensor holds (a complex128 element is two)."""
    if isinstance(x, np.ndarray):
        return int(x.size) * (2 if x.dtype.name == "complex128" else 1)
    return int(x.numel()) * (2 if str(x.dtype).endswith("complex128") else 1)


def _need(x, n: int, name: str):
    """Refuse an array shorter than the n doubles the library will read or write through it."""
    if x is not None and not isinstance(x, int) and _doubles(x) < n:
        raise ValueError(f"{name} holds {_doubles(x)} doubles; this plan needs {n}")


def _c128_interleaved(v) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.complex128))
    return v.view(np.float64).copy()


_KIND = {"dense": ISM_H_DENSE, "bitflip": ISM_H_BITFLIP, "tridiag": ISM_H_TRIDIAG, "gp": ISM_H_GRID_GP,
         "pauli": ISM_H_PAULI}


def pack_hamiltonian(kind: str, H0: np.ndarray, H1: np.ndarray):
    """Dense real-symmetric (H0, H1) -> the packed layout of ism_hkind, checking the structure."""
    H0 = np.asarray(H0, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    d = H0.shape[0]
    if kind == "dense":
        return np.ascontiguousarray(H0).copy(), np.ascontiguousarray(H1).copy()
    if kind == "tridiag":
        for H in (H0, H1):
            if np.any(np.triu(H, 2)) or np.any(np.tril(H, -2)):
                raise ValueError("tridiag kind needs tridiagonal H0 and H1")
        pk = lambda H: np.concatenate([np.diag(H), np.diag(H, 1)]).astype(np.float64)  # noqa: E731
        return pk(H0), pk(H1)
    if kind == "bitflip":
        q = int(round(np.log2(d)))
        if (1 << q) != d:
            raise ValueError("bitflip kind needs d = 2^q")
        if np.any(H0 - np.diag(np.diag(H0))):
            raise ValueError("bitflip kind needs a diagonal H0")
        h = np.array([H1[0, 1 << i] for i in range(q)], dtype=np.float64)
        s = np.arange(d)
        ref = np.zeros((d, d))
        for i in range(q):
            ref[s, s ^ (1 << i)] += h[i]
        if not np.allclose(ref, H1, atol=0.0, rtol=0.0):
            raise ValueError("bitflip kind needs H1 = sum_i h_i X_i")
        return np.diag(H0).astype(np.float64).copy(), h
    raise ValueError(kind)


def measure_peak(which: str = "fp32") -> float:
    """ism_measure_peak: sustained FMA rate of the current GPU in TFLOP/s ("fp32": packed FFMA2, "fp64")."""
    v = C.c_double()
    _check(load().ism_measure_peak({"fp32": 0, "fp64": 1}[which], C.byref(v)))
    return float(v.value)


def subinterval_grad_noalloc(w, precision: str, phi, u, grad, Jn=None, *, batch: int = 1, stream=None,
                             kind: str | None = None):
    """Binding of ism_subinterval_grad_noalloc for callers that cannot allocate device memory: no plan,
    the library uses only its static device scratch; phi, u, grad and Jn must be device buffers."""
    lib = load()
    k = kind or w.kind
    B, Nt, N, d = int(batch), int(w.Nt), int(w.N), int(w.d)
    # the kernels read and write these device buffers in place: refuse short ones
    _need(phi, 2 * B * (N + 1) * d, "phi")
    _need(u, B * Nt, "u")
    _need(grad, B * Nt, "grad")
    _need(Jn, B * N, "Jn")
    prob, _, keep = problem_and_options(w, precision=precision, batch=B, kind=k)   # noqa: F841 (keep alive)
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
    _check(lib.ism_subinterval_grad_noalloc(C.byref(prob), ISM_FP64 if precision == "fp64" else ISM_MIXED,
                                            _ptr(phi), _ptr(u), _ptr(grad), _ptr(Jn), st))


def problem_and_options(w, *, precision=None, batch=1, local_iters=None, rho=None, kind=None, cheb_tol=0.0,
                        subproblem_form=0, step1=0, max_spin_iters=0, scheme="chebyshev", ckpt_stride=0):
    """(ism_problem, ism_options, arrays to keep alive) for a workload object.  scheme: "chebyshev"
    (exact step) or "crank_nicolson" (the Sec. 3 step; FP64, d <= 64, not the grid kinds)."""
    kind = kind or w.kind
    gp = kind == "gp"
    d = int(w.n) if gp else int(w.d)
    prec = precision or w.precision
    dwell = gp and getattr(w, "potential", "harmonic") == "double_well"
    m = 1
    H0i = H1i = None
    if gp:   # grid kinds: H0 = {L, x_min, g} (harmonic trap) or {L, x_min, g, D} (double well)
        H0p = np.array([w.L, w.x_min, w.g] + ([w.dw] if dwell else []), dtype=np.float64)
        H1p = None
    elif kind == "pauli":   # diagonal H0; H1 = [m][q][2] weights (ax, ay)
        m = int(w.m)
        H0p = np.ascontiguousarray(w.H0d, dtype=np.float64)
        H1p = np.ascontiguousarray(np.stack([w.ax, w.ay], axis=-1), dtype=np.float64).reshape(-1)
    elif np.iscomplexobj(w.H0) or np.iscomplexobj(w.H1):   # complex Hermitian: real and imaginary parts
        if kind != "dense":
            raise ValueError("complex H0, H1 are supported for the dense kind only")
        H0p, H1p = pack_hamiltonian(kind, np.real(w.H0), np.real(w.H1))
        H0i = np.ascontiguousarray(np.imag(w.H0), dtype=np.float64)
        H1i = np.ascontiguousarray(np.imag(w.H1), dtype=np.float64)
    else:
        H0p, H1p = pack_hamiltonian(kind, w.H0, w.H1)
    psi_i = _c128_interleaved(w.psi_i)
    psi_f = _c128_interleaved(w.psi_f) if w.objective == "overlap" else None
    O = np.ascontiguousarray(w.O, dtype=np.float64) if w.objective == "observable" else None
    alpha = None if w.alpha is None else np.ascontiguousarray(w.alpha, dtype=np.float64)
    keep = [H0p, H1p, psi_i, psi_f, O, alpha, H0i, H1i]
    prob = IsmProblem(d=d, kind=ISM_H_GRID_GP_DOUBLE_WELL if dwell else _KIND[kind], H0=_ptr(H0p), H1=_ptr(H1p),
                      psi_i=_ptr(psi_i), objective=ISM_OBJ_OVERLAP if w.objective == "overlap" else ISM_OBJ_OBSERVABLE,
                      psi_f=_ptr(psi_f), O=_ptr(O), T=float(w.T), Nt=int(w.Nt), N=int(w.N), alpha=_ptr(alpha),
                      batch=int(batch), controls=m, H0_imag=_ptr(H0i), H1_imag=_ptr(H1i))
    opt = IsmOptions(precision=ISM_FP64 if prec == "fp64" else ISM_MIXED,
                     local_iters=int(local_iters or w.local_iters), rho=float(w.rho if rho is None else rho),
                     cheb_tol=float(cheb_tol), max_spin_iters=int(max_spin_iters),
                     subproblem_form=int(subproblem_form), step1=int(step1), scheme=_SCHEME[scheme],
                     ckpt_stride=int(ckpt_stride))
    return prob, opt, keep


def footprint(w, **kw) -> int:
    """Device bytes a plan for workload w would allocate (ism_plan_footprint; no GPU needed)."""
    prob, opt, keep = problem_and_options(w, **kw)
    n = C.c_size_t()
    _check(load().ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)))
    return int(n.value)


class Plan:
    """An ism_plan over one workload (any object with the fields of workloads.Workload)."""

    def __init__(self, w, *, precision: str | None = None, batch: int = 1, stream=None,
                 local_iters: int | None = None, rho: float | None = None, kind: str | None = None,
                 cheb_tol: float = 0.0, subproblem_form: int = 0, step1: int = 0, max_spin_iters: int = 0,
                 scheme: str = "chebyshev", ckpt_stride: int = 0):
        lib = load()
        self.w = w
        self.kind = kind or w.kind
        self.batch = int(batch)
        self.gp = self.kind == "gp"
        self.m = int(w.m) if self.kind == "pauli" else 1
        self.d = int(w.n) if self.gp else int(w.d)
        self.Nt, self.N = int(w.Nt), int(w.N)
        self.precision = precision or w.precision
        prob, opt, self._keep = problem_and_options(w, precision=precision, batch=batch, local_iters=local_iters,
                                                    rho=rho, kind=kind, cheb_tol=cheb_tol,
                                                    subproblem_form=subproblem_form, step1=step1,
                                                    max_spin_iters=max_spin_iters, scheme=scheme,
                                                    ckpt_stride=ckpt_stride)
        h = C.c_void_p()
        st = None
        if stream is not None:
            st = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
        _check(lib.ism_plan(C.byref(prob), C.byref(opt), st, C.byref(h)))
        self.handle = h

    @classmethod
    def from_problem(cls, prob, opt, keep, stream=None):
        """A plan over a prepared (ism_problem, ism_options) pair (arrays in `keep` stay alive with it)."""
        self = object.__new__(cls)
        self.w = None
        self.kind = {v: k for k, v in _KIND.items()}.get(int(prob.kind), "gp")
        self.batch = max(1, int(prob.batch))
        self.gp = int(prob.kind) in (ISM_H_GRID_GP, ISM_H_GRID_GP_DOUBLE_WELL)
        self.m = max(1, int(prob.controls))
        self.d, self.Nt, self.N = int(prob.d), int(prob.Nt), int(prob.N)
        self.precision = "fp64" if int(opt.precision) == ISM_FP64 else "mixed"
        self._keep = keep
        h = C.c_void_p()
        st = None
        if stream is not None:
            st = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
        _check(load().ism_plan(C.byref(prob), C.byref(opt), st, C.byref(h)))
        self.handle = h
        return self

    # ---------------------------------------------------------------- raw entry points (same names)
    # Each checks that its arrays hold at least the doubles the call reads or writes (layouts of ism.h).
    def _n_u(self) -> int:
        return self.batch * self.Nt * self.m

    def _n_phi(self) -> int:
        return self.batch * (2 if self.gp else 1) * (self.N + 1) * 2 * self.d

    def ism_intermediate_states(self, u, phi):
        _need(u, self._n_u(), "u")
        _need(phi, self._n_phi(), "phi")
        _check(load().ism_intermediate_states(self.handle, _ptr(u), _ptr(phi)))

    def ism_subinterval_grad(self, phi, u, grad, Jn=None):
        _need(phi, self._n_phi(), "phi")
        _need(u, self._n_u(), "u")
        _need(grad, self._n_u(), "grad")
        _need(Jn, self.batch * self.N, "Jn")
        _check(load().ism_subinterval_grad(self.handle, _ptr(phi), _ptr(u), _ptr(grad), _ptr(Jn)))

    def ism_iterate(self, iters, u_inout, J_hist=None, err_hist=None):
        _need(u_inout, self._n_u(), "u_inout")
        _need(J_hist, self.batch * (int(iters) + 1), "J_hist")
        _need(err_hist, self.batch * int(iters), "err_hist")
        _check(load().ism_iterate(self.handle, int(iters), _ptr(u_inout), _ptr(J_hist), _ptr(err_hist)))

    def ism_evaluate(self, u, J=None, F=None):
        _need(u, self._n_u(), "u")
        _need(J, self.batch, "J")
        _need(F, self.batch, "F")
        _check(load().ism_evaluate(self.handle, _ptr(u), _ptr(J), _ptr(F)))

    def ism_gradient(self, u, grad, J=None):
        _need(u, self._n_u(), "u")
        _need(grad, self._n_u(), "grad")
        _need(J, self.batch, "J")
        _check(load().ism_gradient(self.handle, _ptr(u), _ptr(grad), _ptr(J)))

    def ism_set_profiling(self, on: bool):
        _check(load().ism_set_profiling(self.handle, int(bool(on))))

    def ism_get_stats(self, reset: bool = False) -> dict:
        st = IsmStats()
        _check(load().ism_get_stats(self.handle, C.byref(st), int(bool(reset))))
        return {"ms": list(st.ms), "launches": list(st.launches), "y_apps": list(st.y_apps),
                "terms": list(st.terms), "substeps": list(st.substeps), "kernels": int(st.kernels),
                "norm_drift": float(st.norm_drift)}

    def info(self, key: int) -> int:
        return int(load().ism_plan_info(self.handle, key))

    @property
    def ks_large(self) -> bool:
        """True when the global trajectories are propagated directly (d >= 128) instead of assembled."""
        return self.info(5) == 1

    # ---------------------------------------------------------------- numpy conveniences
    def _u(self, u):
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
        return np.ascontiguousarray(np.broadcast_to(u, self._ushape())).copy()

    def _ushape(self):
        """(batch, Nt), or (batch, Nt, m) for several controls."""
        return (self.batch, self.Nt) if self.m == 1 else (self.batch, self.Nt, self.m)

    def _phi_shape(self):
        return (self.batch, 2, self.N + 1, self.d) if self.gp else (self.batch, self.N + 1, self.d)

    def intermediate_states(self, u) -> np.ndarray:
        """phi_n (N+1, d) per problem; for the grid kind the pair sets (2, N+1, d): psi(t_n), chi(t_n)."""
        phi = np.empty(self._phi_shape(), dtype=np.complex128)
        self.ism_intermediate_states(self._u(u), phi.view(np.float64))
        return phi

    def subinterval_grad(self, phi, u):
        phi = np.ascontiguousarray(np.broadcast_to(np.asarray(phi, dtype=np.complex128), self._phi_shape()))
        grad = np.empty(self._ushape())
        Jn = np.empty((self.batch, self.N))
        self.ism_subinterval_grad(phi.view(np.float64), self._u(u), grad, Jn)
        return grad, Jn

    def iterate(self, u, iters: int):
        uu = self._u(u)
        J = np.empty((self.batch, iters + 1))
        E = np.empty((self.batch, max(iters, 1)))
        self.ism_iterate(iters, uu, J, E)
        return uu, J, E[:, :iters]

    def evaluate(self, u):
        J = np.empty(self.batch)
        F = np.empty(self.batch)
        self.ism_evaluate(self._u(u), J, F)
        return J, F

    def gradient(self, u):
        """(dJ/du (batch, Nt) or (batch, Nt, m), J (batch,)) at u."""
        grad = np.empty(self._ushape())
        J = np.empty(self.batch)
        self.ism_gradient(self._u(u), grad, J)
        return grad, J

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().ism_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Serving loop of the C ABI (ism_server_*): concurrent solves of different problems on one GPU,
    admitted by device footprint.  submit() returns a request id; result() waits for it."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 16 << 30, group_capacity: int = 0,
                 group_max_steps: int = 0):
        self.handle = C.c_void_p()
        opt = IsmServerOptions(slots=int(slots), hbm_budget_bytes=int(hbm_budget_bytes),
                               group_capacity=int(group_capacity), group_max_steps=int(group_max_steps))
        rc = load().ism_server_create(C.byref(opt), C.byref(self.handle))
        if rc != ISM_OK:
            raise IsmError(rc, "ism_server_create")
        self._shape = {}

    def submit_problem(self, prob, opt, u0, iters: int) -> int:
        """Submit a prepared (ism_problem, ism_options) pair for one problem; u0: (Nt,) controls."""
        u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64)).reshape(1, -1)
        _need(u, int(prob.Nt), "u0")
        rid = C.c_longlong()
        _check(load().ism_server_submit(self.handle, C.byref(prob), C.byref(opt), _ptr(u), int(iters), C.byref(rid)))
        self._shape[rid.value] = ((1, int(prob.Nt)), int(iters))
        return rid.value

    def submit(self, w, u0=None, iters=None, batch: int = 1, **plan_kw) -> int:
        prob, opt, keep = problem_and_options(w, batch=batch, **plan_kw)
        Nt = int(w.Nt)
        ushape = (batch, Nt, int(w.m)) if getattr(w, "kind", "") == "pauli" else (batch, Nt)
        u = np.ascontiguousarray(np.broadcast_to(np.asarray(w.u0 if u0 is None else u0, dtype=np.float64),
                                                 ushape)).copy()
        it = int(w.iters if iters is None else iters)
        rid = C.c_longlong()
        _check(load().ism_server_submit(self.handle, C.byref(prob), C.byref(opt), _ptr(u), it, C.byref(rid)))
        self._shape[rid.value] = (ushape, it)
        return rid.value

    def poll(self, rid: int, wait: bool = False):
        """(state, u (batch, Nt[, m]) or None, J_hist (batch, iters+1) or None, times_ms (3,))."""
        ushape, it = self._shape[rid]
        st = C.c_int()
        u = np.empty(ushape)
        J = np.empty((ushape[0], it + 1))
        t = np.empty(3)
        _check(load().ism_server_poll(self.handle, C.c_longlong(rid), int(bool(wait)), C.byref(st), _ptr(u), _ptr(J),
                                      _ptr(t)))
        done = st.value == ISM_REQ_DONE
        return st.value, (u if done else None), (J if done else None), t

    def stats(self) -> dict:
        """ism_server_stats: shared passes, request-passes they carried, most requests in one pass,
        shared plans opened, requests run on their own plans."""
        out = (C.c_longlong * 5)()
        _check(load().ism_server_stats(self.handle, out))
        return {"passes": out[0], "request_passes": out[1], "max_rows": out[2], "groups": out[3], "single": out[4]}

    def result(self, rid: int):
        st, u, J, t = self.poll(rid, wait=True)
        load().ism_server_release(self.handle, C.c_longlong(rid))
        self._shape.pop(rid, None)
        return u, J, t

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().ism_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
