"""libexpd builds, loads and exports every symbol include/expd.h declares; the
host-side argument checks and the FFT / preconditioner index arithmetic are
exercised without a GPU (no compute call reaches the device here)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from paper_2603_04350_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def expd():
    B.build()
    from paper_2603_04350_gb300 import expd as E
    E.lib()
    return E


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(expd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("expd_plan_create", "expd_residual", "expd_precond_apply", "expd_solve_fp",
                     "expd_solve_gmres", "expd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(expd):
    lib = expd.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(expd.SYMBOLS) <= declared_functions()


def test_host_selftest_fft_and_preconditioner():
    exe = B.build_selftest()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")


def _spec(expd, **kw):
    base = dict(bc=expd.BC_PERIODIC, n=(16, 16), length=(1.0, 1.0), a=0.01, c=0.0, nonlin=expd.NL_NONE,
                dt=0.01, Nt=8, alpha=0.01, order=1)
    base.update(kw)
    return expd.PlanSpec(**base)


def test_plan_create_rejects_too_long_windows_without_touching_the_gpu(expd):
    with pytest.raises(expd.ExpdError) as ei:
        expd.plan_create(_spec(expd, n=(16,), length=(1.0,), Nt=514, order=2))   # Ns = 513
    assert ei.value.status == expd.ERR_UNSUPPORTED and "512" in str(ei.value)


@pytest.mark.parametrize("kw,msg", [
    (dict(alpha=1.5), "alpha"),
    (dict(alpha=0.0), "alpha"),
    (dict(dt=-1.0), "dt"),
    (dict(order=7), "order"),
    (dict(order=3, Nt=3), "Nt"),
    (dict(n=(12, 16)), "powers of two"),
    (dict(n=(4, 16)), "powers of two"),
    (dict(bc=1, n=(1, 5)), "Dirichlet"),
    (dict(nonlin=1, dt=2.0), "beta_s*dt"),
    (dict(tol=0.0), "tol"),
    (dict(max_iter=0), "max_iter"),
    (dict(gmres_restart=0), "gmres_restart"),
    (dict(precision=7), "precision"),
    (dict(n=(8, 8, 8)), "ndim"),
    (dict(bc=1, n=(7, 7), b=(0.5, 0.0)), "advection needs a periodic grid"),
    (dict(jacobian=5), "jacobian"),
    (dict(guess=3), "guess"),
    (dict(a=0.01 + 1j), "complex_state"),
    (dict(c=2j), "complex_state"),
])
def test_plan_create_rejects_bad_arguments_without_touching_the_gpu(expd, kw, msg):
    spec = _spec(expd, **kw)
    if len(spec.n) > 2:
        g = expd.Grid()
        g.ndim = 3
        h = C.c_void_p()
        st = expd.lib().expd_plan_create(C.byref(g), C.byref(expd.Operator(0.01, 0.0, 0)), 0.01, 8, 0.01,
                                         C.byref(expd.Scheme(1, 0, 10, 1e-8, 20, 0)), None, C.byref(h))
        assert st == expd.ERR_INVALID_ARG and not h.value
        return
    with pytest.raises(expd.ExpdError) as ei:
        expd.plan_create(spec)
    assert ei.value.status == expd.ERR_INVALID_ARG
    assert msg in str(ei.value)


@pytest.mark.parametrize("kw,msg", [
    (dict(a=1j, c=2j, complex_state=True, precision=1), "float64"),
    (dict(a=1j, complex_state=True, nonlin=1), "linear"),
])
def test_plan_create_rejects_unbuilt_complex_state_cases_without_touching_the_gpu(expd, kw, msg):
    with pytest.raises(expd.ExpdError) as ei:
        expd.plan_create(_spec(expd, **kw))
    assert ei.value.status == expd.ERR_UNSUPPORTED and msg in str(ei.value)


def test_every_entry_point_has_declared_argument_types(expd):
    # ctypes passes undeclared pointer arguments as 32-bit ints; every entry
    # point that takes arguments must declare them
    lib = expd.lib()
    for name in expd.SYMBOLS:
        if name in ("expd_last_error", "expd_version"):
            continue
        assert getattr(lib, name).argtypes, name


def test_null_arguments_are_rejected(expd):
    lib = expd.lib()
    assert lib.expd_destroy(None) == expd.OK
    assert lib.expd_solve_fp(None, None, None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_residual(None, None, None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_precond_apply(None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_solve_gmres(None, None, None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_solve_bicgstab(None, None, None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_solve_sequential(None, None, None, None, None) == expd.ERR_INVALID_ARG
    assert lib.expd_timing_enable(None, 1) == expd.ERR_INVALID_ARG
    assert lib.expd_status_string(3) == b"not converged"
    assert lib.expd_version() >= 10000


def test_kernel_classes_match_the_header(expd):
    # the binding's timing struct and class names follow the header's enum
    text = open(os.path.join(ROOT, "include", "expd.h")).read()
    n = int(re.search(r"EXPD_NUM_KCLASS\s*=\s*(\d+)", text).group(1))
    assert expd.NUM_KCLASS == n == len(expd.KCLASS_NAMES)
    enum = {m.group(1): int(m.group(2)) for m in re.finditer(r"EXPD_K_(\w+)\s*=\s*(\d+)", text)}
    assert sorted(enum.values()) == list(range(n))
    assert enum["DST_TC"] == expd.KCLASS_NAMES.index("dst_tc") == expd.K_DST_TC
    assert enum["DST_SPLIT"] == expd.KCLASS_NAMES.index("dst_split") == expd.K_DST_SPLIT
    assert C.sizeof(expd.Timing) == C.sizeof(C.c_longlong) + n * (C.sizeof(C.c_int) + 3 * C.sizeof(C.c_double)) + \
        (4 if (n * C.sizeof(C.c_int)) % 8 else 0)
