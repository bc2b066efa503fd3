"""Checkpoint and resume (marked gpu): with EXPD_GUESS_GIVEN every solver starts
from the iterate the caller passes in U (its unknown slices u_s..u_Nt), e.g. the
last iterate of a call that stopped at max_iter, a time limit or a cancel,
kept in device memory or copied to the host and back.

The fixed point's next iterate from a checkpoint matches the oracle's sweep
from the same iterate (Eq. (3.2), the float64 bar); GMRES and BiCGStab resumed
from a checkpoint reach the sequential solution (Sec. 7's norm, 1e-10), and a
resume from the solution itself stops at once.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def expd():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd as E
    return E


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def P(name, bc, n, order, Nt, nonlin="none", a=0.01, c=0.1, dt=0.01, alpha=1e-2):
    return I.Problem(name=name, bc=bc, n=tuple(n), length=tuple(1.0 for _ in n), a=a, c=c, nonlin=nonlin, dt=dt,
                     Nt=Nt, alpha=alpha, order=order)


CASES = [
    P("dir2d_s2", "dirichlet", (13, 11), 2, Nt=20),
    P("dir1d_s6_tc", "dirichlet", (300,), 6, Nt=40, alpha=1e-3, dt=1e-3),
    P("per2d_s1", "periodic", (16, 32), 1, Nt=24),
    P("neu2d_s3", "neumann", (12, 10), 3, Nt=18),
]
IDS = [p.name for p in CASES]
NL = P("per2d_ac_s2", "periodic", (16, 16), 2, Nt=21, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, alpha=1e-3)


def inputs(p, seed):
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    return u0, f


@pytest.mark.parametrize("p", CASES + [NL], ids=IDS + [NL.name])
def test_fp_sweep_from_a_checkpoint_matches_oracle(expd, p):
    sp = O.spec_of(p)
    u0, f = inputs(p, 1)
    fd = None if f is None else dev(f)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-300, max_iter=2)) as plan:
        info = plan.solve_fp(dev(u0), fd, U, allow_not_converged=True)
    assert info["iterations"] == 2
    ckpt = host(U)  # the checkpoint, through host memory
    U2 = torch.from_numpy(ckpt.copy()).to(DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-300, max_iter=1, guess=expd.GUESS_GIVEN)) as plan:
        info = plan.solve_fp(dev(u0), fd, U2, allow_not_converged=True)
    assert info["iterations"] == 1
    ref = O.richardson(sp, u0, f, max_iter=1, V0=ckpt[p.order - 1:]).U[1:]
    assert O.rel_error(host(U2), ref) < 1e-12
    # the same as three sweeps in one call
    U3 = torch.empty_like(U)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-300, max_iter=3)) as plan:
        plan.solve_fp(dev(u0), fd, U3, allow_not_converged=True)
    assert O.rel_error(host(U2), host(U3)) < 1e-12


@pytest.mark.parametrize("p", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("solver", ["gmres", "bicgstab", "fp"])
def test_resumed_solve_reaches_the_solution(expd, p, prec, solver):
    sp = O.spec_of(p)
    u0, f = inputs(p, 2)
    seq = O.sequential_solve(sp, u0, f)[1:]
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=1)) as plan:
        getattr(plan, "solve_" + solver)(dev(u0), dev(f), U, allow_not_converged=True)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=300,
                                                 guess=expd.GUESS_GIVEN)) as plan:
        info = getattr(plan, "solve_" + solver)(dev(u0), dev(f), U)  # U in place: the device checkpoint
    assert O.rel_error(host(U), seq) < 1e-10, info


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
def test_resume_from_the_solution_stops_at_once(expd, solver):
    p = CASES[0]
    u0, f = inputs(p, 3)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=300)) as plan:
        first = getattr(plan, "solve_" + solver)(dev(u0), dev(f), U)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=300, guess=expd.GUESS_GIVEN)) as plan:
        again = getattr(plan, "solve_" + solver)(dev(u0), dev(f), U)
    assert first["iterations"] > 1
    assert again["iterations"] <= 1, again


def test_resume_from_host_pointers(expd):
    p = CASES[0]
    sp = O.spec_of(p)
    u0, f = inputs(p, 4)
    seq = O.sequential_solve(sp, u0, f)[1:]
    U = np.zeros((p.Nt,) + p.n)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=1)) as plan:
        plan.solve_gmres(np.ascontiguousarray(u0), np.ascontiguousarray(f), U, allow_not_converged=True)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=300, guess=expd.GUESS_GIVEN)) as plan:
        plan.solve_gmres(np.ascontiguousarray(u0), np.ascontiguousarray(f), U)
    assert O.rel_error(U, seq) < 1e-10
