"""Autotuner on the GPU (marked gpu): every candidate is timed, the fastest is
kept, and a plan created with it solves to the same result as the default
plan (both against the oracle's sequential solution)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import autotune, expd
    return autotune, expd


@pytest.mark.parametrize("p", [I.ALLEN_CAHN_256.with_(n=(64, 64), Nt=16, tol=1e-10),
                               I.HEAT_DIRICHLET_1024.with_(n=(128, 256), Nt=9, dt=0.1 / 9, tol=1e-10)],
                         ids=["periodic_64x64_nt16", "dirichlet_128x256_nt9"])
def test_tuned_plan_matches_default(mods, p):
    A, expd = mods
    tuner = A.Tuner(reps=2, warmup=1)
    entry = tuner.tune(p, expd.PREC_MIXED)
    assert len(entry["trials"]) == len(A.candidates(p, expd.PREC_MIXED)) >= 2
    assert all(t["ms"] > 0 for t in entry["trials"])
    assert entry["ms"] == min(t["ms"] for t in entry["trials"])
    u0, f = I.make_inputs(p)
    ref = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, max_iter=200)
    fd = None if f is None else torch.from_numpy(f).to(DEV)
    for make in (lambda: tuner.plan_create(p, spec), lambda: expd.plan_create(spec)):
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with make() as plan:
            (plan.solve_gmres if p.solver == "gmres" else plan.solve_fp)(torch.from_numpy(u0).to(DEV), fd, U)
        torch.cuda.synchronize()
        assert O.rel_error(U.cpu().numpy(), ref) < 1e-9
