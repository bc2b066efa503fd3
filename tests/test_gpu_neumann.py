"""Neumann grids on the GPU (zero normal derivative, cell-centred 3/5-point
Laplacian, DCT-II eigenbasis; the Allen-Cahn experiment of Sec. 7) against
the oracle, through the C ABI (marked gpu).

The float64 path is held to 1e-11 element-wise for single operations and to
1e-10 in Sec. 7's error norm for solves at tol 1e-12; the mixed path's
preconditioner to the float32 bound eps32/alpha, its solves to the same
1e-10 (the refinement and the accurate sweeps reach the float64 fixed point).
"""
import math

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


def dev(x, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def P(name, n, order, nonlin="none", a=0.05, c=0.1, Nt=None, alpha=1e-2, dt=0.01):
    return I.Problem(name=name, bc="neumann", n=tuple(n), length=tuple(1.0 for _ in n), a=a, c=c, nonlin=nonlin,
                     dt=dt, Nt=Nt if Nt is not None else order + 9, alpha=alpha, order=order)


# several time-kernel tiles with ragged tails; Ns = 29 is a Bluestein window
CASES = [
    P("n1_s1", (64,), 1),
    P("n1_s6", (50,), 6, Nt=17),
    P("n2_s2", (15, 31), 2),
    P("n2_blue_s2", (9, 13), 2, Nt=30),
    P("n2_ac_s1", (24, 20), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, alpha=1e-3),
    P("n2_ac_s2", (16, 12), 2, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, alpha=1e-3),
]
IDS = [p.name for p in CASES]
LINEAR = [p for p in CASES if p.nonlin == "none"]
LIN_IDS = [p.name for p in LINEAR]


@pytest.mark.parametrize("p", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neumann_precond_apply(expd, p, prec):
    r = np.random.default_rng(1).standard_normal((p.Ns,) + p.n)
    ref = O.precond_apply(O.spec_of(p), r)
    S = torch.empty_like(dev(r))
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    with expd.plan_create(expd.spec_from_problem(p, precision=precision)) as plan:
        plan.precond_apply(dev(r), S)
    bound = 1e-11 if prec == "fp64" else 6e-8 * 16 / p.alpha
    assert relmax(host(S), ref) < bound


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_neumann_residual(expd, p):
    sp = O.spec_of(p)
    rng = np.random.default_rng(3)
    amp = 0.5 if p.nonlin != "none" else 1.0
    u0 = amp * rng.uniform(-1, 1, p.n)
    U = amp * rng.uniform(-1, 1, (p.Nt,) + p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    U_start = np.concatenate([u0[None], U[: p.order - 1]])
    ref = O.residual(sp, U[p.order - 1:], O.rhs_known(sp, U_start, f))
    R = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.residual(dev(u0), dev(f), dev(U), R)
    assert relmax(host(R), ref) < 1e-11


@pytest.mark.parametrize("p", LINEAR, ids=LIN_IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neumann_linear_solvers_match_sequential(expd, p, prec):
    sp = O.spec_of(p)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    seq = O.sequential_solve(sp, u0, f)[1:]
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=300)) as plan:
        plan.solve_sequential(dev(u0), dev(f), U)
        assert O.rel_error(host(U), seq) < 1e-12
        for fn in (plan.solve_gmres, plan.solve_bicgstab, plan.solve_fp):
            U.zero_()
            fn(dev(u0), dev(f), U)
            assert O.rel_error(host(U), seq) < 1e-10, fn.__name__


@pytest.mark.parametrize("p", [c for c in CASES if c.nonlin != "none"], ids=["ac_s1", "ac_s2"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neumann_allen_cahn_fixed_point(expd, p, prec):
    sp = O.spec_of(p)
    u0 = np.random.default_rng(7).uniform(-0.9, 0.9, p.n)
    seq = O.sequential_solve(sp, u0)[1:]
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=300)) as plan:
        plan.solve_fp(dev(u0), None, U)
        assert O.rel_error(host(U), seq) < 1e-10
        plan.solve_sequential(dev(u0), None, U)
        assert O.rel_error(host(U), seq) < 1e-12


@pytest.mark.parametrize("p", [CASES[2], CASES[4]], ids=[IDS[2], IDS[4]])
def test_neumann_richardson_iterates_match_oracle(expd, p):
    # per-iteration parity of the fixed point from the linear initial iterate
    sp = O.spec_of(p)
    u0 = np.random.default_rng(9).uniform(-0.8, 0.8, p.n)
    for k in (1, 2, 3):
        ref = O.richardson(sp, u0, None, max_iter=k, init="linear").U[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, tol=1e-300, max_iter=k)) as plan:
            info = plan.solve_fp(dev(u0), None, U, allow_not_converged=True)
        assert info["iterations"] == k
        assert O.rel_error(host(U), ref) < 1e-12


def test_neumann_allen_cahn_exact_solution(expd):
    # Sec. 7's Neumann Allen-Cahn problem (eps = 0.01, exact solution
    # 0.5 e^{-t} cos(2 pi x) through a manufactured source): the GPU solve
    # agrees with the oracle's sequential solution and its error against the
    # exact solution halves with dt (first order)
    eps, n, T = 0.01, 256, 0.1
    errs = []
    for Nt in (25, 50):
        dt = T / Nt
        p = I.Problem(name="ac_neumann_exact", bc="neumann", n=(n,), length=(1.0,), a=eps**2, c=0.0,
                      nonlin="allen_cahn", dt=dt, Nt=Nt, alpha=1e-3, order=1, tol=1e-12)
        x = I.grid_coords(p)[0]

        def ue(t):
            return 0.5 * np.exp(-t) * np.cos(2 * np.pi * x)
        f = np.array([ue((k + 1) * dt) * (4 * np.pi**2 * eps**2 - 2) + ue((k + 1) * dt) ** 3 for k in range(Nt)])
        U = torch.empty((Nt, n), dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, max_iter=200)) as plan:
            plan.solve_fp(dev(ue(0.0)), dev(f), U)
        got = host(U)
        seq = O.sequential_solve(O.spec_of(p), ue(0.0), f)[1:]
        assert O.rel_error(got, seq) < 1e-10
        errs.append(O.rel_error(got, np.array([ue((k + 1) * dt) for k in range(Nt)])))
    assert abs(errs[0] / errs[1] - 2.0) < 0.2


def test_neumann_complex_state(expd):
    p = I.Problem(name="se_neumann", bc="neumann", n=(12, 10), length=(1.0, 1.0), a=1j, c=2j, nonlin="none",
                  dt=0.01, Nt=12, alpha=1e-2, order=2, complex_state=True)
    sp = O.spec_of(p)
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    seq = O.sequential_solve(sp, u0)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=100)) as plan:
        plan.solve_gmres(dev(u0, np.complex128), None, U)
    assert O.rel_error(host(U), seq) < 1e-10


def test_neumann_footprint_matches_allocation(expd):
    for p, prec in ((CASES[2], expd.PREC_FP64), (CASES[4], expd.PREC_MIXED)):
        spec = expd.spec_from_problem(p, precision=prec)
        with expd.plan_create(spec) as plan:
            assert plan.workspace_bytes() == expd.plan_footprint_bytes(spec), p.name
