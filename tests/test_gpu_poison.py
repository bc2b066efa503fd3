"""Debug modes on the GPU (marked gpu): solves with every plan buffer filled
with NaN bytes at allocation, and with guard words after every buffer.

EXPD_POISON=1 makes the library fill each new device buffer with all-ones
bytes, a NaN in every floating type.  A kernel that reads a buffer (or a part
of one) before writing it then turns the solution non-finite, whatever the
memory held before; without the fill such a read sees whatever an earlier
allocation left there and fails only in long-running processes.  The cases
are the served mix's Dirichlet requests, every (N_t, s) the mix draws at two
grids (one through the dense sine transform, one through the FFT-based one),
the float64 and the mixed path, against the oracle's sequential solution
(Sec. 7's error norm at the workload's tolerance).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")

MIX_NT = (16, 32, 64, 128, 256)
MIX_ORDERS = (1, 2, 6)


@pytest.fixture(scope="module")
def expd():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd as E
    return E


def _case(g, nt, s):
    return I.HEAT_DIRICHLET_1024.with_(name=f"heat_{g}_{nt}_{s}", n=(g, g), Nt=nt, dt=0.1 / nt, order=s)


_SEQ = {}


def _sequential(p):
    key = (p.n, p.Nt, p.order)
    if key not in _SEQ:
        u0, f = I.make_inputs(p)
        _SEQ[key] = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    return _SEQ[key]


@pytest.mark.parametrize("g", (64, 63))
@pytest.mark.parametrize("nt", MIX_NT)
@pytest.mark.parametrize("s", MIX_ORDERS)
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_poisoned_buffers_dirichlet_gmres(expd, monkeypatch, g, nt, s, prec):
    monkeypatch.setenv("EXPD_POISON", "1")
    p = _case(g, nt, s)
    u0, f = I.make_inputs(p)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200)) as plan:
        # twice on one plan: the second solve starts from the buffers the first left
        for _ in range(2):
            U.fill_(float("nan"))
            plan.solve_gmres(torch.from_numpy(u0).to(DEV), torch.from_numpy(f).to(DEV), U)
            torch.cuda.synchronize()
            out = U.cpu().numpy()
            assert np.isfinite(out).all()
            assert O.rel_error(out, _sequential(p)) < p.tol


@pytest.mark.parametrize("solver", ("fp", "bicgstab", "sequential"))
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_poisoned_buffers_other_solvers(expd, monkeypatch, solver, prec):
    monkeypatch.setenv("EXPD_POISON", "1")
    p = _case(63, 64, 2)
    u0, f = I.make_inputs(p)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.full((p.Nt,) + p.n, float("nan"), dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200)) as plan:
        fn = {"fp": plan.solve_fp, "bicgstab": plan.solve_bicgstab, "sequential": plan.solve_sequential}[solver]
        fn(torch.from_numpy(u0).to(DEV), torch.from_numpy(f).to(DEV), U)
        torch.cuda.synchronize()
    out = U.cpu().numpy()
    assert np.isfinite(out).all()
    assert O.rel_error(out, _sequential(p)) < p.tol


@pytest.mark.parametrize("order", (1, 6))
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_poisoned_buffers_allen_cahn(expd, monkeypatch, order, prec):
    monkeypatch.setenv("EXPD_POISON", "1")
    base = I.ALLEN_CAHN_512_S6 if order == 6 else I.ALLEN_CAHN_256
    p = base.with_(n=(64, 64), Nt=32)
    u0 = I.make_u0(p)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.full((p.Nt,) + p.n, float("nan"), dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200)) as plan:
        plan.solve_fp(torch.from_numpy(u0).to(DEV), None, U)
        torch.cuda.synchronize()
    out = U.cpu().numpy()
    assert np.isfinite(out).all()
    assert O.rel_error(out, O.sequential_solve(O.spec_of(p), u0)[1:]) < p.tol


# EXPD_CANARY=1 puts 256 guard bytes after every workspace buffer and checks
# them after each solver call: no kernel writes past the end of a buffer.
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
@pytest.mark.parametrize("solver", ("gmres", "bicgstab", "fp"))
def test_canary_guard_words_stay_intact_dirichlet(expd, monkeypatch, prec, solver):
    monkeypatch.setenv("EXPD_CANARY", "1")
    p = I.HEAT_DIRICHLET_1024.with_(n=(256, 256), Nt=32, dt=0.1 / 32)      # tensor-core sine transforms (mixed)
    u0, f = I.make_inputs(p)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200)) as plan:
        fn = {"gmres": plan.solve_gmres, "bicgstab": plan.solve_bicgstab, "fp": plan.solve_fp}[solver]
        fn(torch.from_numpy(u0).to(DEV), torch.from_numpy(f).to(DEV), U)
    assert O.rel_error(U.cpu().numpy(), _sequential(p)) < p.tol


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_canary_guard_words_stay_intact_allen_cahn(expd, monkeypatch, prec):
    monkeypatch.setenv("EXPD_CANARY", "1")
    p = I.ALLEN_CAHN_512_S6.with_(n=(64, 64), Nt=40)
    u0 = I.make_u0(p)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200)) as plan:
        plan.solve_fp(torch.from_numpy(u0).to(DEV), None, U)
    assert O.rel_error(U.cpu().numpy(), O.sequential_solve(O.spec_of(p), u0)[1:]) < p.tol


def test_canary_guard_words_stay_intact_complex_state(expd, monkeypatch):
    monkeypatch.setenv("EXPD_CANARY", "1")
    p = I.SCHRODINGER_2D.with_(Nt=20)
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, max_iter=50)) as plan:
        plan.solve_gmres(torch.from_numpy(u0).to(DEV), None, U)
    assert O.rel_error(U.cpu().numpy(), O.sequential_solve(O.spec_of(p), u0, f)[1:]) < 1e-10
