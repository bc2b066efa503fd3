"""The allocation-free preconditioner entry point (expd_precond_apply_noalloc).

It serves callers that cannot allocate device memory (their memory is owned by
an allocator of their own, or an allocation could fail or stall mid-run): it
keeps all of its tables and intermediates in one fixed device array.  Its
output must equal the plan-based expd_precond_apply's on the same input,
within the float64 parity tolerance the other preconditioner tests use, on two
calls in a row (two different problems, so a stale array from the first call
cannot mask an error in the second).  The mixed-precision cases run the
register time kernel (16, 32 and 64 unknown slices) with the array's smaller
norm-partial grid and are held to the float32 preconditioner's bound against
both the plan path and the oracle; a Dirichlet size with n + 1 a power of two
checks the array's dense sine products against the plan's FFT-based ones.
This file is collected last.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expd():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd as E
    return E


def _problems():
    return [
        I.Problem(name="noalloc_periodic", bc="periodic", n=(32, 64), length=(1.0, 1.0), a=0.01, c=0.1,
                  nonlin="none", dt=0.01, Nt=16, alpha=1e-2, order=2),            # Ns = 15, Bluestein
        I.Problem(name="noalloc_dirichlet", bc="dirichlet", n=(13, 11), length=(1.0, 1.0), a=0.01, c=0.1,
                  nonlin="none", dt=0.01, Nt=16, alpha=1e-2, order=1),            # Ns = 16, radix-2
    ]


def test_noalloc_precond_matches_plan_path_on_two_calls(expd):
    dev = torch.device("cuda:0")
    for k, p in enumerate(_problems()):
        spec = expd.spec_from_problem(p)
        R = torch.from_numpy(np.random.default_rng(10 + k).standard_normal((p.Ns,) + p.n)).to(dev)
        S_plan = torch.empty_like(R)
        with expd.plan_create(spec) as plan:
            plan.precond_apply(R, S_plan)
        S_free = torch.full_like(R, math.nan)
        expd.precond_apply_noalloc(spec, R, S_free)
        torch.cuda.synchronize()
        a, b = S_free.cpu().numpy(), S_plan.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-11, p.name


def test_noalloc_rejects_problems_beyond_its_array(expd):
    p = I.ALLEN_CAHN_256.with_(nonlin="none")
    R = torch.zeros((p.Ns,) + p.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(expd.ExpdError) as ei:
        expd.precond_apply_noalloc(expd.spec_from_problem(p), R, R)
    assert ei.value.status == expd.ERR_INVALID_ARG
    assert "bytes of scratch" in str(ei.value)


def _mixed_problems():
    # Ns = Nt - s + 1 in {16, 32, 64}: the register time kernel with the
    # float32 preconditioner, periodic and Dirichlet, orders 1 and 2
    out = []
    for ns, bc, order in ((16, "periodic", 1), (32, "dirichlet", 2), (64, "periodic", 2)):
        n = (16, 64) if bc == "periodic" else (13, 23)
        out.append(I.Problem(name=f"noalloc_mixed_{bc}_ns{ns}", bc=bc, n=n, length=(1.0, 1.0), a=0.01,
                             c=0.1, nonlin="none", dt=1e-3, Nt=ns + order - 1, alpha=1e-3, order=order))
    return out


@pytest.mark.parametrize("p", _mixed_problems(), ids=lambda p: p.name)
def test_noalloc_mixed_register_kernel_matches_plan_and_oracle(expd, p):
    dev = torch.device("cuda:0")
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED)
    r = np.random.default_rng(21).standard_normal((p.Ns,) + p.n)
    R = torch.from_numpy(r).to(dev)
    S_plan = torch.empty_like(R)
    with expd.plan_create(spec) as plan:
        plan.precond_apply(R, S_plan)
    outs = []
    for _ in range(2):  # two calls in a row on the shared array
        S_free = torch.full_like(R, math.nan)
        expd.precond_apply_noalloc(spec, R, S_free)
        torch.cuda.synchronize()
        outs.append(S_free.cpu().numpy())
    ref = O.precond_apply(O.spec_of(p), r)
    bound = 6e-8 * 16 / p.alpha  # float32 steps (a)-(c): eps32 * log2(L) / alpha relative
    b = S_plan.cpu().numpy()
    for a in outs:
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() / np.abs(b).max() < bound, p.name
        assert np.abs(a - ref).max() / np.abs(ref).max() < bound, p.name
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_dirichlet_fast_dst_size_matches_plan(expd):
    # n + 1 a power of two: the plan transforms with odd-extension FFTs, the
    # allocation-free call with the dense sine matrices it builds in the array
    dev = torch.device("cuda:0")
    p = I.Problem(name="noalloc_fast_dst", bc="dirichlet", n=(15, 7), length=(1.0, 1.0), a=0.01, c=0.1,
                  nonlin="none", dt=0.01, Nt=12, alpha=1e-2, order=2)
    spec = expd.spec_from_problem(p)
    r = np.random.default_rng(22).standard_normal((p.Ns,) + p.n)
    R = torch.from_numpy(r).to(dev)
    S_plan = torch.empty_like(R)
    with expd.plan_create(spec) as plan:
        plan.precond_apply(R, S_plan)
    S_free = torch.full_like(R, math.nan)
    expd.precond_apply_noalloc(spec, R, S_free)
    torch.cuda.synchronize()
    a, b = S_free.cpu().numpy(), S_plan.cpu().numpy()
    ref = O.precond_apply(O.spec_of(p), r)
    assert np.abs(a - b).max() / np.abs(b).max() < 1e-11
    assert np.abs(a - ref).max() / np.abs(ref).max() < 1e-11


def test_noalloc_clears_the_last_error(expd):
    # a failing call leaves its message; the next successful call clears it
    p = _problems()[0]
    spec = expd.spec_from_problem(p)
    R = torch.zeros((p.Ns,) + p.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(expd.ExpdError):
        expd.precond_apply_noalloc(expd.spec_from_problem(I.ALLEN_CAHN_256.with_(nonlin="none")), R, R)
    assert expd.lib().expd_last_error().decode() != ""
    expd.precond_apply_noalloc(spec, R, R)
    torch.cuda.synchronize()
    assert expd.lib().expd_last_error().decode() == ""
