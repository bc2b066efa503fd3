"""The allocation-free preconditioner entry point (expd_precond_apply_noalloc).

It serves callers that cannot allocate device memory (their memory is owned by
an allocator of their own, or an allocation could fail or stall mid-run): it
keeps all of its tables and intermediates in one fixed device array.  Its
output must equal the plan-based expd_precond_apply's on the same input,
within the float64 parity tolerance the other preconditioner tests use, on two
calls in a row (two different problems, so a stale array from the first call
cannot mask an error in the second).  This file is collected last.
"""
import math

import numpy as np
import pytest
import torch

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
