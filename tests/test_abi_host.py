"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry point
that include/ism.h declares, and rejects malformed problems before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1603_01237_gb300 import abi

    return abi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ism.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ism_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ism_plan", "ism_intermediate_states", "ism_subinterval_grad", "ism_iterate", "ism_plan_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_1603_01237_gb300 import abi

    assert set(abi.EXPORTS) <= set(declared_functions())


def test_version(lib):
    assert b"sm_103a" in lib.ism_version()


def _problem(abi, **kw):
    d = kw.pop("d", 4)
    H0 = kw.pop("H0", np.zeros(d * d))
    H1 = kw.pop("H1", np.eye(d).ravel())
    psi = np.zeros(2 * d)
    psi[0] = 1.0
    base = dict(d=d, kind=abi.ISM_H_DENSE, H0=H0.ctypes.data, H1=H1.ctypes.data, psi_i=psi.ctypes.data,
                objective=abi.ISM_OBJ_OVERLAP, psi_f=psi.ctypes.data, O=None, T=1.0, Nt=10, N=2, alpha=None,
                batch=1)
    base.update(kw)
    keep = (H0, H1, psi)
    return abi.IsmProblem(**base), keep


@pytest.mark.parametrize("field,value,status", [
    ("d", 0, 1), ("Nt", 0, 1), ("N", 0, 1), ("N", 11, 1), ("T", 0.0, 1), ("T", float("nan"), 1),
    ("kind", 7, 1), ("objective", 5, 1), ("psi_f", None, 1), ("batch", -1, 1), ("d", 65, 6),
])
def test_plan_rejects_bad_problems(lib, field, value, status):
    from paper_1603_01237_gb300 import abi

    prob, keep = _problem(abi)
    setattr(prob, field, value)
    opt = abi.IsmOptions(precision=0, local_iters=1, rho=0.1, cheb_tol=0.0, max_spin_iters=0, subproblem_form=0)
    h = C.c_void_p()
    rc = lib.ism_plan(C.byref(prob), C.byref(opt), None, C.byref(h))
    assert rc == status
    assert h.value is None
    assert len(lib.ism_last_error()) > 0


def test_plan_rejects_nonsymmetric_and_nonfinite(lib):
    from paper_1603_01237_gb300 import abi

    opt = abi.IsmOptions(precision=0, local_iters=1, rho=0.1, cheb_tol=0.0, max_spin_iters=0, subproblem_form=0)
    H0 = np.arange(16.0)
    prob, keep = _problem(abi, H0=H0)
    h = C.c_void_p()
    assert lib.ism_plan(C.byref(prob), C.byref(opt), None, C.byref(h)) == abi.ISM_EINVAL
    H0 = np.zeros(16)
    H0[5] = np.inf
    prob, keep = _problem(abi, H0=H0)
    assert lib.ism_plan(C.byref(prob), C.byref(opt), None, C.byref(h)) == abi.ISM_ENONFINITE
    bad = abi.IsmOptions(precision=3, local_iters=1, rho=0.1, cheb_tol=0.0, max_spin_iters=0, subproblem_form=0)
    prob, keep = _problem(abi)
    assert lib.ism_plan(C.byref(prob), C.byref(bad), None, C.byref(h)) == abi.ISM_EINVAL


def test_bitflip_needs_power_of_two(lib):
    from paper_1603_01237_gb300 import abi

    prob, keep = _problem(abi, d=6, kind=abi.ISM_H_BITFLIP, H0=np.zeros(6), H1=np.ones(3))
    opt = abi.IsmOptions(precision=0, local_iters=1, rho=0.1, cheb_tol=0.0, max_spin_iters=0, subproblem_form=0)
    h = C.c_void_p()
    assert lib.ism_plan(C.byref(prob), C.byref(opt), None, C.byref(h)) == abi.ISM_EINVAL


@pytest.mark.parametrize("kind_name", ["ISM_H_BITFLIP", "ISM_H_PAULI"])
@pytest.mark.parametrize("d,status", [(2 ** 31 - 1, 1), (2 ** 30 + 1, 1), (2 ** 30, 6), (2048, 6)])
def test_power_of_two_kinds_reject_huge_d(lib, kind_name, d, status):
    """The kinds with d = 2^q take q from d on the host; a d near the int range must give an error
    (not a power of two: ISM_EINVAL; a power of two above 1024: ISM_EUNSUPPORTED), before any array
    of that size is read."""
    from paper_1603_01237_gb300 import abi

    prob, keep = _problem(abi, kind=getattr(abi, kind_name))
    prob.d = d
    opt = abi.IsmOptions(precision=0, local_iters=1, rho=0.1, cheb_tol=0.0, max_spin_iters=0, subproblem_form=0)
    n = C.c_size_t()
    assert lib.ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)) == status
    assert len(lib.ism_last_error()) > 0


def test_noalloc_entry_point_refuses_other_kinds_on_the_host(lib):
    """The allocation-free entry point runs the Chebyshev sweep of the dense, tridiagonal and bit-flip
    layouts: a grid problem (H0 = three grid parameters, no H1) or a Pauli problem is refused before
    any array is read or any device memory is touched."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    gp = W.gp_bec(n=64, Nt=40, N=4, steps=50)
    pauli = W.random_pauli(7, 2, 5, T=1.0, Nt=40, N=4)
    dummy = np.zeros(2 * 2 * 5 * 128)
    for w in (gp, pauli):
        prob, opt, keep = abi.problem_and_options(w, precision="fp64")
        rc = lib.ism_subinterval_grad_noalloc(C.byref(prob), 0, dummy.ctypes.data, dummy.ctypes.data,
                                              dummy.ctypes.data, None, None)
        assert rc == abi.ISM_EUNSUPPORTED
        assert "dense, tridiagonal and bit-flip" in lib.ism_last_error().decode()


def test_binding_accepts_only_double_arrays():
    """The C ABI reads every array as doubles: the binding refuses narrower element types (which the
    library would read past their end) and non-contiguous data, host or torch."""
    import torch

    from paper_1603_01237_gb300 import abi

    assert abi._ptr(None) is None
    assert abi._ptr(np.zeros(4)) > 0
    assert abi._ptr(np.zeros(4, dtype=np.complex128)) > 0
    assert abi._ptr(torch.zeros(4, dtype=torch.float64)) > 0
    assert abi._ptr(torch.zeros(4, dtype=torch.complex128)) > 0
    for bad in (np.zeros(4, dtype=np.float32), np.zeros(4, dtype=np.int64), np.zeros(4, dtype=np.complex64),
                torch.zeros(4, dtype=torch.float32), torch.zeros(4, dtype=torch.int32)):
        with pytest.raises(TypeError):
            abi._ptr(bad)
    with pytest.raises(ValueError):
        abi._ptr(np.zeros((4, 4))[:, 0])
    with pytest.raises(ValueError):
        abi._ptr(torch.zeros(4, 4, dtype=torch.float64).t())


@pytest.mark.parametrize("gp,m", [(False, 1), (True, 1), (False, 3)])
def test_plan_methods_refuse_short_arrays(lib, gp, m):
    """The raw Plan methods pass bare pointers, so each first checks that every array holds the doubles
    ism.h's layout gives it ([batch][Nt](*m) controls and gradients, [batch](*2)*(N+1)*2d states,
    [batch][iters+1] and [batch][iters] histories); a short array is refused before the library is
    called (no plan is needed for that: this one has no handle)."""
    from paper_1603_01237_gb300 import abi

    pl = object.__new__(abi.Plan)
    pl.handle, pl.batch, pl.Nt, pl.N, pl.d, pl.gp, pl.m = None, 3, 20, 4, 8, gp, m
    nu, nphi = 3 * 20 * m, 3 * (2 if gp else 1) * 5 * 2 * 8
    u, g, phi = np.zeros(nu), np.zeros(nu), np.zeros(nphi)
    short = lambda n: np.zeros(n - 1)   # noqa: E731
    cases = [
        lambda: pl.ism_intermediate_states(short(nu), phi),
        lambda: pl.ism_intermediate_states(u, short(nphi)),
        lambda: pl.ism_intermediate_states(u, np.zeros(nphi // 2 - 1, dtype=np.complex128)),
        lambda: pl.ism_subinterval_grad(phi, u, short(nu)),
        lambda: pl.ism_subinterval_grad(phi, u, g, short(3 * 4)),
        lambda: pl.ism_iterate(5, short(nu)),
        lambda: pl.ism_iterate(5, u, short(3 * 6)),
        lambda: pl.ism_iterate(5, u, None, short(3 * 5)),
        lambda: pl.ism_evaluate(u, short(3)),
        lambda: pl.ism_gradient(u, short(nu)),
    ]
    for call in cases:
        with pytest.raises(ValueError):
            call()
    # arrays of the right size reach the library, which refuses the missing plan
    with pytest.raises(abi.IsmError):
        pl.ism_subinterval_grad(np.zeros(nphi // 2, dtype=np.complex128), u, g, np.zeros(3 * 4))


def test_null_arguments(lib):
    from paper_1603_01237_gb300 import abi

    h = C.c_void_p()
    assert lib.ism_plan(None, None, None, C.byref(h)) == abi.ISM_EINVAL
    assert lib.ism_iterate(None, 1, None, None, None) == abi.ISM_EINVAL
    assert lib.ism_intermediate_states(None, None, None) == abi.ISM_EINVAL
    assert lib.ism_subinterval_grad(None, None, None, None, None) == abi.ISM_EINVAL
    assert lib.ism_plan_destroy(None) == abi.ISM_OK
    assert lib.ism_plan_info(None, 0) == -1


def test_pack_hamiltonian_checks_structure():
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41", Nt=10, N=2)
    H0p, H1p = abi.pack_hamiltonian("tridiag", w.H0, w.H1)
    assert H0p.shape == (2 * w.d - 1,) and np.allclose(H1p[:w.d], 0.0)
    with pytest.raises(ValueError):
        abi.pack_hamiltonian("bitflip", w.H0, w.H1)
    s = W.config("spin16", Nt=10, N=2)
    d0, h = abi.pack_hamiltonian("bitflip", s.H0, s.H1)
    assert np.allclose(h, 1.0) and np.allclose(d0, np.diag(s.H0))
    with pytest.raises(ValueError):
        abi.pack_hamiltonian("tridiag", s.H0, s.H1)


def test_footprint_needs_no_gpu_and_scales_with_the_problem(lib):
    """ism_plan_footprint sizes a plan on the host: it grows linearly with the batch and with Nt,
    and rejects what ism_plan rejects."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41", Nt=2000, N=16)
    f1 = abi.footprint(w, batch=1)
    f2 = abi.footprint(w, batch=2)
    f4 = abi.footprint(w, batch=4)
    assert 0 < f1 < f2 < f4
    assert abs((f4 - f2) - 2 * (f2 - f1)) <= 8 * 512   # per-problem part, up to allocation rounding
    assert abi.footprint(W.config("rotor41", Nt=4000, N=16)) > f1
    # d = 1024: the sub-problems store no per-step states (first local steps recompute both trajectories
    # from the partition, literal ones checkpoint), so 18000 more steps add per-step scalars, not states
    f_short, f_long = abi.footprint(W.config("ising1024", Nt=2000, N=16)), abi.footprint(W.config("ising1024", Nt=20000, N=16))
    assert 0 < f_long - f_short < 18000 * 1024 * 8 / 50
    f_lit = abi.footprint(W.config("ising1024", Nt=20000, N=16), precision="fp64")
    assert f_lit - abi.footprint(W.config("ising1024", Nt=2000, N=16), precision="fp64") < 18000 * 1024 * 16 / 5
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(W.config("rotor41", Nt=100, N=200))
    assert ei.value.status == 1


def test_crank_nicolson_option_validated_on_the_host(lib):
    """The Crank-Nicolson scheme is accepted in both precisions for the tridiagonal, dense and bit-flip
    kinds with d <= 64; its plans hold none of the per-step trajectories of the concurrent
    two-trajectory sweeps (its first local steps run both trajectories forward in one group)."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41", Nt=2000, N=16)
    f_cn = abi.footprint(w, precision="mixed", scheme="crank_nicolson", step1=1)
    f_ch = abi.footprint(w, precision="mixed", step1=1)
    assert 0 < f_cn < f_ch
    assert abi.footprint(w, precision="mixed", scheme="crank_nicolson") > 0   # FP32 Cayley steps
    assert abi.footprint(W.random_dense(5, 3, T=1.0, Nt=50, N=2), scheme="crank_nicolson") > 0
    assert abi.footprint(W.config("spin16", Nt=100), scheme="crank_nicolson") > 0
    for big in (W.config("ising1024", Nt=200, N=4), W.gp_bec(n=64, Nt=20, N=2, steps=10)):
        with pytest.raises(abi.IsmError) as ei:
            abi.footprint(big, precision="fp64", scheme="crank_nicolson")
        assert ei.value.status == abi.ISM_EUNSUPPORTED
    prob, opt, keep = abi.problem_and_options(w, precision="fp64")
    opt.scheme = 7
    n = abi.C.c_size_t()
    assert lib.ism_plan_footprint(abi.C.byref(prob), abi.C.byref(opt), abi.C.byref(n)) == abi.ISM_EINVAL


def test_several_controls_validated_on_the_host(lib):
    """The Pauli kind (several controls): sized per control, d = 128..1024 only, overlap objective, no
    penalty; the controls field is refused on the other kinds."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.random_pauli(8, 3, 7, T=1.0, Nt=100, N=4)
    f3 = abi.footprint(w, precision="mixed")
    f1 = abi.footprint(w.with_(ax=w.ax[:1], ay=w.ay[:1], u0=w.u0[:, :1]), precision="mixed")
    assert f3 > f1 > 0   # controls, gradients per control
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(W.random_pauli(6, 2, 7, T=1.0, Nt=50, N=2))
    assert ei.value.status == abi.ISM_EUNSUPPORTED   # d = 64: the Pauli kind needs d >= 128
    prob, opt, keep = abi.problem_and_options(w, precision="fp64")
    n = abi.C.c_size_t()
    prob.controls = 33
    assert lib.ism_plan_footprint(abi.C.byref(prob), abi.C.byref(opt), abi.C.byref(n)) == abi.ISM_EINVAL
    s = W.config("spin16", Nt=100)
    prob, opt, keep = abi.problem_and_options(s, precision="fp64")
    prob.controls = 2
    assert lib.ism_plan_footprint(abi.C.byref(prob), abi.C.byref(opt), abi.C.byref(n)) == abi.ISM_EINVAL
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(w, precision="fp64", scheme="crank_nicolson")
    assert ei.value.status == abi.ISM_EUNSUPPORTED


def test_double_well_kind_validated_on_the_host(lib):
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.gp_double_well(n=64, Nt=50, N=2, steps=10)
    assert abi.footprint(w) > 0
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(w.with_(dw=-1.0))
    assert ei.value.status == abi.ISM_EINVAL


def test_server_validates_options_requests_and_ids_on_the_host(lib):
    """The serving loop's host-side checks (ism_server_*): bad options, a request larger than the
    whole budget, unknown request ids; nothing here reaches the device."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    for slots, budget in ((0, 1 << 30), (65, 1 << 30), (2, 0)):
        with pytest.raises(abi.IsmError) as ei:
            abi.Server(slots=slots, hbm_budget_bytes=budget)
        assert ei.value.status == abi.ISM_EINVAL
    with abi.Server(slots=2, hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(abi.IsmError) as ei:      # footprint + history + slack > 1 MiB
            srv.submit(W.config("rotor41", Nt=2000, N=16), iters=2)
        assert ei.value.status == abi.ISM_ENOMEM and "budget" in str(ei.value)
        st = C.c_int()
        assert lib.ism_server_poll(srv.handle, C.c_longlong(12345), 0, C.byref(st), None, None, None) == abi.ISM_EINVAL
        assert b"unknown request id" in lib.ism_last_error()
        assert lib.ism_server_release(srv.handle, C.c_longlong(12345)) == abi.ISM_EINVAL


def test_server_reports_a_failed_request_without_a_gpu(lib):
    """With no CUDA device the request is admitted, its plan fails in the worker, and poll() returns
    the plan's error: the failure travels back through the queue instead of hanging or aborting."""
    import torch

    import workloads as W
    from paper_1603_01237_gb300 import abi

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the request would run (covered by the GPU serving tests)")
    with abi.Server(slots=2, hbm_budget_bytes=1 << 30) as srv:
        rid = srv.submit(W.config("spin16", Nt=100, N=4), iters=1)
        with pytest.raises(abi.IsmError) as ei:
            srv.poll(rid, wait=True)
        assert ei.value.status == abi.ISM_ECUDA
        state = C.c_int()
        lib.ism_server_poll(srv.handle, C.c_longlong(rid), 0, C.byref(state), None, None, None)
        assert state.value == abi.ISM_REQ_FAILED
        assert lib.ism_server_release(srv.handle, C.c_longlong(rid)) == abi.ISM_OK


def test_noalloc_binding_refuses_short_arrays():
    """The allocation-free entry point reads and writes the caller's device buffers in place as
    [batch][N+1][2d], [batch][Nt], [batch][Nt] and [batch][N]: the binding refuses a short one before
    the library is called."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41", Nt=120, N=6)
    B, nphi, nu = 3, 2 * 3 * 7 * 41, 3 * 120
    ok = dict(phi=np.zeros(nphi), u=np.zeros(nu), grad=np.zeros(nu), Jn=np.zeros(3 * 6))
    for name, n in (("phi", nphi), ("u", nu), ("grad", nu), ("Jn", 3 * 6)):
        args = dict(ok)
        args[name] = np.zeros(n - 1)
        with pytest.raises(ValueError, match=name):
            abi.subinterval_grad_noalloc(w, "mixed", args["phi"], args["u"], args["grad"], args["Jn"], batch=B)


def test_checkpoint_stride_sets_the_literal_footprint(lib):
    """ckpt_stride S: a literal sub-problem holds ceil(n_steps/S) states and S vectors H1 psi per (problem,
    n), never its whole trajectory; a plan whose first local steps run the two-trajectory form (the
    default in both precisions) stores no states and holds neither unless L > 1.  Negative strides
    are refused."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41")                       # Nt = 20000, N = 128: 157 steps per sub-interval
    B, GE, N = 64, 48, 128                        # the sub-interval sweep holds 16 lanes x 3 elements
    fp = lambda **kw: abi.footprint(w, batch=B, step1=2, **kw)   # noqa: E731
    base = fp(precision="mixed")
    for S in (1, 13, 157):
        nck = -(-157 // S)
        lit = B * N * (nck * 2 * GE * 8 + S * GE * 8)            # FP32 hi + lo checkpoints, segment
        got = fp(precision="mixed", local_iters=2, ckpt_stride=S) - base
        assert abs(got - lit) <= 2 * 512, (S, got, lit)
    traj = B * (20000 + N) * GE * 8                               # a whole per-step trajectory
    assert fp(precision="mixed", local_iters=2) - base < traj / 4   # ~3 sqrt(n_steps) vectors vs n_steps
    prob, opt, keep = abi.problem_and_options(w, precision="fp64", ckpt_stride=-1)
    n = C.c_size_t()
    assert lib.ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)) == abi.ISM_EINVAL


def test_complex_hermitian_dense_validated_on_the_host(lib):
    """Imaginary parts: the dense kind only, antisymmetric, finite, d <= 64, Chebyshev scheme; the
    complex plan stages both parts of H (a larger op array than the real plan's)."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.random_hermitian(24, 5, T=1.0, Nt=60, N=3)
    fc = abi.footprint(w, precision="fp64")
    fr = abi.footprint(w.with_(H0=w.H0.real.copy(), H1=w.H1.real.copy()), precision="fp64")
    assert fc > fr > 0
    assert abi.footprint(w, precision="mixed") > 0
    assert abi.footprint(w.with_(objective="observable", psi_f=None, O=np.eye(24)), precision="fp64") > 0
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(w, precision="fp64", scheme="crank_nicolson")
    assert ei.value.status == abi.ISM_EUNSUPPORTED
    n = C.c_size_t()
    opt = abi.IsmOptions(precision=0, local_iters=1, rho=0.1)
    for bad_imag, status in ((np.ones((24, 24)), abi.ISM_EINVAL),              # not antisymmetric
                             (np.diag(np.ones(24)), abi.ISM_EINVAL),           # diagonal must vanish
                             (np.full((24, 24), np.nan), abi.ISM_ENONFINITE)):
        prob, _, keep = abi.problem_and_options(w, precision="fp64")
        bad = np.ascontiguousarray(bad_imag, dtype=np.float64)
        prob.H1_imag = bad.ctypes.data
        assert lib.ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)) == status
    prob, _, keep = abi.problem_and_options(W.config("rotor41", Nt=100, N=4), precision="fp64")
    im = np.zeros(100)
    prob.H0_imag = im.ctypes.data                                             # tridiagonal kind
    assert lib.ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)) == abi.ISM_EINVAL
    big = W.random_hermitian(128, 6, T=1.0, Nt=20, N=2)                       # the tensor-core sizes are real only
    with pytest.raises(abi.IsmError) as ei:
        abi.footprint(big, precision="mixed")
    assert ei.value.status == abi.ISM_EUNSUPPORTED


def test_grid_kind_checkpoints_size_the_plan(lib):
    """Grid kinds: ckpt_stride 0 stores the whole forward trajectory; S > 0 stores every S-th state
    of each sub-interval and one segment per sub-problem, so the footprint falls with S up to
    ~sqrt(steps per sub-interval)."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.gp_double_well(n=512, Nt=10000, N=64, steps=200)
    f = {S: abi.footprint(w, precision="fp64", ckpt_stride=S) for S in (0, 1, 4, 13, 157)}
    assert f[13] < f[4] < f[1] and f[13] < f[157] and f[13] < 0.25 * f[0]
    n = C.c_size_t()
    prob, opt, keep = abi.problem_and_options(w, precision="fp64", ckpt_stride=-1)
    assert lib.ism_plan_footprint(C.byref(prob), C.byref(opt), C.byref(n)) == abi.ISM_EINVAL


def test_fp64_first_local_steps_default_to_the_two_trajectory_form(lib):
    """FP64 plans run a first local step in the two-trajectory form, as mixed ones do: the default
    FP64 plan holds no literal checkpoints, and asking for the literal form (subproblem_form 1) or a
    second local step adds them (one state every S steps and an S-step segment per (problem, n))."""
    import workloads as W
    from paper_1603_01237_gb300 import abi

    w = W.config("rotor41")                       # Nt = 20000, N = 128
    fp = lambda **kw: abi.footprint(w, batch=64, step1=2, precision="fp64", **kw)   # noqa: E731
    default, two, literal, local2 = fp(), fp(subproblem_form=2), fp(subproblem_form=1), fp(local_iters=2)
    assert default == two
    assert literal > default and local2 > default
    assert literal - default > 64 * 128 * 41 * 16   # at least one FP64 complex state per (problem, n)
