"""Device buffers that are not 16-byte aligned (marked gpu).

A torch view that starts at an odd float64 element has an 8-byte-aligned data
pointer.  The kernels read 16-byte vectors and copy 16-byte-aligned rows in
bulk, so the library stages such buffers through its own device buffers (as
it stages host buffers): the results are bit for bit those of aligned buffers
holding the same values.  The allocation-free entry point cannot stage and
refuses them on the host, before any kernel runs.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

from .test_gpu_parity import DEV, P, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expd():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd as E
    return E


def odd_view(x):
    """A copy of x in device memory whose data pointer is 8 (mod 16)."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    buf = torch.empty(a.size + 1, dtype=torch.float64, device=DEV)
    v = buf[1:].view(a.shape)
    v.copy_(torch.from_numpy(a))
    assert v.data_ptr() % 16 == 8
    return v


def odd_empty(shape):
    n = int(np.prod(shape))
    buf = torch.full((n + 1,), np.nan, dtype=torch.float64, device=DEV)
    v = buf[1:].view(shape)
    assert v.data_ptr() % 16 == 8
    return v


CASES = [
    # tensor-core DST (digit split with bulk-staged rows), float32 time kernels
    P("tc_dir_256x128_s2", "dirichlet", (256, 128), 2, Nt=10),
    # periodic FFTs
    P("per_64x32_s1", "periodic", (64, 32), 1, Nt=12),
    # fast DST-I (n + 1 a power of two), odd total sizes
    P("dir_15x7_s3", "dirichlet", (15, 7), 3, Nt=9),
]
IDS = [p.name for p in CASES]


@pytest.mark.parametrize("p", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_precond_apply_unaligned_equals_aligned(expd, p, prec):
    precision = expd.PREC_MIXED if prec == "mixed" else expd.PREC_FP64
    r = np.random.default_rng(1).standard_normal((p.Ns,) + p.n)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision)) as plan:
        S_a = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
        plan.precond_apply(dev(r), S_a)
        S_u = odd_empty((p.Ns,) + p.n)
        plan.precond_apply(odd_view(r), S_u)
    assert np.array_equal(host(S_u), host(S_a))


@pytest.mark.parametrize("p", CASES, ids=IDS)
@pytest.mark.parametrize("solver", ["gmres", "fp"])
def test_solve_unaligned_equals_aligned(expd, p, solver):
    rng = np.random.default_rng(2)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=300)
    with expd.plan_create(spec) as plan:
        U_a = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        getattr(plan, "solve_" + solver)(dev(u0), dev(f), U_a)
        U_u = odd_empty((p.Nt,) + p.n)
        getattr(plan, "solve_" + solver)(odd_view(u0), odd_view(f), U_u)
    got = host(U_u)
    assert np.array_equal(got, host(U_a))
    seq = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    assert O.rel_error(got, seq) < 1e-10


def test_residual_unaligned_equals_aligned(expd):
    p = CASES[0]
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, p.n)
    U = rng.uniform(-1, 1, (p.Nt,) + p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10)) as plan:
        R_a = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
        plan.residual(dev(u0), dev(f), dev(U), R_a)
        R_u = odd_empty((p.Ns,) + p.n)
        plan.residual(odd_view(u0), odd_view(f), odd_view(U), R_u)
    assert np.array_equal(host(R_u), host(R_a))


def test_noalloc_refuses_unaligned_buffers(expd):
    p = CASES[1]
    r = np.random.default_rng(4).standard_normal((p.Ns,) + p.n)
    spec = expd.spec_from_problem(p)
    S = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
    with pytest.raises(expd.ExpdError) as e:
        expd.precond_apply_noalloc(spec, odd_view(r), S)
    assert e.value.status == expd.ERR_INVALID_ARG
    assert "aligned" in str(e.value)
    # the aligned call still works afterwards
    expd.precond_apply_noalloc(spec, dev(r), S)
    torch.cuda.synchronize()
    assert np.isfinite(host(S)).all()
