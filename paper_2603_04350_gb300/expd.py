"""Thin ctypes binding of libexpd (include/expd.h): argument marshalling only.

Every function keeps the C name without the `expd_` prefix.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays, float64 and C-contiguous; the
library itself detects host versus device pointers.  Nothing here computes:
a missing or unloadable libexpd.so raises instead of falling back to Python.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libexpd.so")

(OK, ERR_INVALID_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT,
 ERR_CANCELLED) = range(9)
BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
NL_NONE, NL_ALLEN_CAHN = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
STARTUP_RAMP, STARTUP_GIVEN = 0, 1
JAC_LAGGED, JAC_MEAN_U0 = 0, 1
GUESS_LINEAR, GUESS_ZERO, GUESS_GIVEN = 0, 1, 2
KF_TIME_SMEM, KF_FFT_RADIX4, KF_DST_FP64, KF_DST_N64 = 1, 2, 4, 8
NLF_IF, NLF_ETD1 = 0, 1
MAX_HISTORY = 128

SYMBOLS = ("expd_plan_create", "expd_plan_workspace_bytes", "expd_plan_footprint_bytes", "expd_residual", "expd_precond_apply",
           "expd_solve_fp", "expd_solve_gmres", "expd_solve_bicgstab", "expd_solve_sequential", "expd_plan_cancel",
           "expd_timing_enable", "expd_timing_read", "expd_destroy",
           "expd_precond_apply_noalloc",
           "expd_status_string", "expd_last_error", "expd_version")
(K_TIME, K_FFT_COL, K_FFT_ROW, K_DST, K_GMRES, K_POINTWISE, K_REDUCE, K_TIME32, K_FFT_COL32, K_FFT_ROW32,
 K_TIMEDD, K_FFT_COLDD, K_FFT_ROWDD, K_DST_TC, K_DST_SPLIT, K_TIME_TC) = range(16)
NUM_KCLASS = 16
KCLASS_NAMES = ("time", "fft_col", "fft_row", "dst", "gmres", "pointwise", "reduce", "time32", "fft_col32",
                "fft_row32", "timedd", "fft_coldd", "fft_rowdd", "dst_tc", "dst_split", "time_tc")


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 2), ("length", C.c_double * 2), ("bc", C.c_int)]


class Operator(C.Structure):
    _fields_ = [("a", C.c_double), ("c", C.c_double), ("nonlin", C.c_int), ("b", C.c_double * 2),
                ("a_im", C.c_double), ("c_im", C.c_double), ("complex_state", C.c_int)]


class Scheme(C.Structure):
    _fields_ = [("order", C.c_int), ("precision", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double),
                ("gmres_restart", C.c_int), ("startup", C.c_int), ("jacobian", C.c_int), ("guess", C.c_int),
                ("kernel_flags", C.c_int), ("nl_form", C.c_int), ("time_limit_ms", C.c_double)]


class Info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("fp32_iterations", C.c_int), ("final_measure", C.c_double),
                ("contraction", C.c_double), ("history", C.c_double * MAX_HISTORY), ("refinements", C.c_int),
                ("ms_setup", C.c_double), ("ms_iterate", C.c_double), ("ms_output", C.c_double)]

    def as_dict(self):
        k = max(0, min(self.iterations + 1, MAX_HISTORY))
        return {"iterations": self.iterations, "fp32_iterations": self.fp32_iterations,
                "final_measure": self.final_measure, "contraction": self.contraction,
                "history": [self.history[i] for i in range(k)], "refinements": self.refinements,
                "ms_setup": self.ms_setup, "ms_iterate": self.ms_iterate, "ms_output": self.ms_output}


class Timing(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("count", C.c_int * NUM_KCLASS), ("ms", C.c_double * NUM_KCLASS),
                ("bytes", C.c_double * NUM_KCLASS), ("flops", C.c_double * NUM_KCLASS)]

    def as_dict(self):
        return {"launches": self.launches,
                "classes": {KCLASS_NAMES[i]: {"count": self.count[i], "ms": self.ms[i], "bytes": self.bytes[i],
                                              "flops": self.flops[i]} for i in range(NUM_KCLASS)}}


class ExpdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"expd status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libexpd.so (built in-tree by paper_2603_04350_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libexpd.so not built ({LIB_PATH}); run paper_2603_04350_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.c_void_p
    L.expd_plan_create.argtypes = [C.POINTER(Grid), C.POINTER(Operator), C.c_double, C.c_int, C.c_double,
                                   C.POINTER(Scheme), vp, C.POINTER(vp)]
    L.expd_plan_workspace_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
    L.expd_plan_footprint_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Operator), C.c_double, C.c_int, C.c_double,
                                            C.POINTER(Scheme), C.c_int, C.POINTER(C.c_size_t)]
    L.expd_residual.argtypes = [vp, dp, dp, dp, dp, vp]
    L.expd_precond_apply.argtypes = [vp, dp, dp, vp]
    L.expd_solve_fp.argtypes = [vp, dp, dp, dp, C.POINTER(Info), vp]
    L.expd_solve_gmres.argtypes = [vp, dp, dp, dp, C.POINTER(Info), vp]
    L.expd_solve_sequential.argtypes = [vp, dp, dp, dp, vp]
    L.expd_solve_bicgstab.argtypes = [vp, dp, dp, dp, C.POINTER(Info), vp]
    L.expd_plan_cancel.argtypes = [vp]
    L.expd_timing_enable.argtypes = [vp, C.c_int]
    L.expd_timing_read.argtypes = [vp, C.POINTER(Timing), C.c_int]
    L.expd_destroy.argtypes = [vp]
    L.expd_precond_apply_noalloc.argtypes = [C.POINTER(Grid), C.POINTER(Operator), C.c_double, C.c_int,
                                             C.c_double, C.POINTER(Scheme), dp, dp, vp]
    L.expd_status_string.argtypes = [C.c_int]
    L.expd_status_string.restype = C.c_char_p
    L.expd_last_error.restype = C.c_char_p
    L.expd_version.restype = C.c_int
    for name in SYMBOLS:
        if name not in ("expd_status_string", "expd_last_error", "expd_version"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int, allow=(OK,)) -> int:
    if status not in allow:
        raise ExpdError(status, lib().expd_last_error().decode() or lib().expd_status_string(status).decode())
    return status


def _ptr(x, cplx: bool = False) -> Optional[int]:
    """Data pointer of a C-contiguous torch tensor or numpy array: float64, or
    complex128 (interleaved re, im doubles) for a plan with a complex state."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        want = np.complex128 if cplx else np.float64
        if x.dtype != want or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"arrays must be {np.dtype(want).name} and C-contiguous")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        want = torch.complex128 if cplx else torch.float64
        if x.dtype != want or not x.is_contiguous():
            raise ValueError(f"tensors must be {want} and contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class PlanSpec:
    bc: int
    n: tuple
    length: tuple
    a: float
    c: float
    nonlin: int
    dt: float
    Nt: int
    alpha: float
    order: int
    precision: int = PREC_FP64
    max_iter: int = 100
    tol: float = 1e-8
    gmres_restart: int = 20
    startup: int = STARTUP_RAMP
    jacobian: int = 0
    b: tuple = (0.0, 0.0)
    guess: int = GUESS_LINEAR
    kernel_flags: int = 0
    nl_form: int = NLF_IF
    time_limit_ms: float = 0.0
    complex_state: bool = False   # complex a, c and complex128 state arrays


def _structs(spec: PlanSpec):
    g = Grid()
    g.ndim = len(spec.n)
    for d in range(g.ndim):
        g.n[d] = int(spec.n[d])
        g.length[d] = float(spec.length[d])
    g.bc = spec.bc
    a, c = complex(spec.a), complex(spec.c)
    o = Operator(a.real, c.real, spec.nonlin, (C.c_double * 2)(*(tuple(spec.b) + (0.0, 0.0))[:2]),
                 a.imag, c.imag, 1 if spec.complex_state else 0)
    s = Scheme(spec.order, spec.precision, spec.max_iter, spec.tol, spec.gmres_restart, spec.startup, spec.jacobian,
               spec.guess, spec.kernel_flags, spec.nl_form, spec.time_limit_ms)
    return g, o, s


FOOTPRINT_SOURCE, FOOTPRINT_HOST, FOOTPRINT_GMRES = 1, 2, 4


def plan_footprint_bytes(spec: PlanSpec, flags: int = 0) -> int:
    """Device bytes plan_create(spec) would allocate (plus lazily allocated
    buffers selected by flags), computed without allocating."""
    g, o, s = _structs(spec)
    b = C.c_size_t()
    _check(lib().expd_plan_footprint_bytes(C.byref(g), C.byref(o), spec.dt, spec.Nt, spec.alpha, C.byref(s),
                                           int(flags), C.byref(b)))
    return b.value


def precond_apply_noalloc(spec: PlanSpec, R, S, stream=None) -> None:
    """expd_precond_apply_noalloc: the preconditioner solve without a plan and
    without any device allocation (R, S device tensors)."""
    g, o, s = _structs(spec)
    _check(lib().expd_precond_apply_noalloc(C.byref(g), C.byref(o), spec.dt, spec.Nt, spec.alpha, C.byref(s),
                                            _ptr(R), _ptr(S), _stream(stream)))


def plan_create(spec: PlanSpec, stream=None) -> "Plan":
    g, o, s = _structs(spec)
    h = C.c_void_p()
    _check(lib().expd_plan_create(C.byref(g), C.byref(o), spec.dt, spec.Nt, spec.alpha, C.byref(s),
                                  _stream(stream), C.byref(h)))
    return Plan(h, spec)


class Plan:
    """Owner of an expd_plan handle; the methods map one-to-one onto the C ABI."""

    def __init__(self, handle: C.c_void_p, spec: PlanSpec):
        self._h = handle
        self.spec = spec
        self.Ns = spec.Nt - spec.order + 1
        self._c = bool(spec.complex_state)

    def _p(self, x):
        return _ptr(x, self._c)

    def workspace_bytes(self) -> int:
        b = C.c_size_t()
        _check(lib().expd_plan_workspace_bytes(self._h, C.byref(b)))
        return b.value

    def residual(self, u0, f, U, R, stream=None) -> None:
        _check(lib().expd_residual(self._h, self._p(u0), self._p(f), self._p(U), self._p(R), _stream(stream)))

    def precond_apply(self, R, S, stream=None) -> None:
        _check(lib().expd_precond_apply(self._h, self._p(R), self._p(S), _stream(stream)))

    def solve_fp(self, u0, f, U, stream=None, allow_not_converged=False) -> dict:
        info = Info()
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        st = _check(lib().expd_solve_fp(self._h, self._p(u0), self._p(f), self._p(U), C.byref(info), _stream(stream)),
                    allow)
        d = info.as_dict()
        d["status"] = st
        return d

    def solve_gmres(self, u0, f, U, stream=None, allow_not_converged=False) -> dict:
        info = Info()
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        st = _check(lib().expd_solve_gmres(self._h, self._p(u0), self._p(f), self._p(U), C.byref(info),
                                           _stream(stream)),
                    allow)
        d = info.as_dict()
        d["status"] = st
        return d

    def solve_bicgstab(self, u0, f, U, stream=None, allow_not_converged=False) -> dict:
        info = Info()
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        st = _check(lib().expd_solve_bicgstab(self._h, self._p(u0), self._p(f), self._p(U), C.byref(info),
                                              _stream(stream)),
                    allow)
        d = info.as_dict()
        d["status"] = st
        return d

    def cancel(self) -> None:
        """expd_plan_cancel: stop the call in flight on this plan (or its next one)."""
        _check(lib().expd_plan_cancel(self._h))

    def solve_sequential(self, u0, f, U, stream=None) -> None:
        """Step the scheme sequentially (float64): the exact all-at-once solution."""
        _check(lib().expd_solve_sequential(self._h, self._p(u0), self._p(f), self._p(U), _stream(stream)))

    def timing_enable(self, enable: bool = True) -> None:
        _check(lib().expd_timing_enable(self._h, 1 if enable else 0))

    def timing_read(self, reset: bool = True) -> dict:
        t = Timing()
        _check(lib().expd_timing_read(self._h, C.byref(t), 1 if reset else 0))
        return t.as_dict()

    def destroy(self) -> None:
        if self._h:
            lib().expd_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spec_from_problem(p, precision: int = PREC_FP64, max_iter: int = 100, tol: Optional[float] = None,
                      gmres_restart: int = 20, startup: int = STARTUP_RAMP, jacobian: int = 0,
                      guess: int = GUESS_LINEAR, kernel_flags: int = 0, nl_form: Optional[int] = None,
                      time_limit_ms: float = 0.0) -> PlanSpec:
    """PlanSpec from a paper_2603_04350_gb300.inputs.Problem."""
    bc = {"periodic": BC_PERIODIC, "dirichlet": BC_DIRICHLET, "neumann": BC_NEUMANN}[p.bc]
    return PlanSpec(bc=bc, n=tuple(p.n), length=tuple(p.length),
                    a=p.a, c=p.c, nonlin=NL_ALLEN_CAHN if p.nonlin == "allen_cahn" else NL_NONE, dt=p.dt,
                    Nt=p.Nt, alpha=p.alpha, order=p.order, precision=precision, max_iter=max_iter,
                    tol=p.tol if tol is None else tol, gmres_restart=gmres_restart, startup=startup,
                    jacobian=jacobian, b=tuple(getattr(p, "b", ()) or (0.0, 0.0)), guess=guess,
                    kernel_flags=kernel_flags,
                    nl_form=(NLF_ETD1 if getattr(p, "nl_form", "if") == "etd1" else NLF_IF) if nl_form is None
                    else nl_form, time_limit_ms=time_limit_ms,
                    complex_state=bool(getattr(p, "complex_state", False)))
