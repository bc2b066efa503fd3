"""Complex states on the GPU (the Schrodinger equation of Sec. 7) against the
oracle, through the C ABI (marked gpu).

L = (a + i a_im) Lap - (c + i c_im) with complex128 arrays: the spatial
transforms act on real and imaginary parts alike (complex FFTs on periodic
grids, the sine transform of both parts on Dirichlet grids), the time kernel
takes complex columns with a complex symbol, GMRES runs in complex arithmetic.
The float64 parity bar is 1e-11 element-wise for single operations and 1e-10
in Sec. 7's error norm for solves at tol 1e-12.
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cfield(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def P(name, bc, n, order, a=1j, c=2j, Nt=None, alpha=1e-2, dt=0.01):
    length = tuple(2 * math.pi if bc == "periodic" else 1.0 for _ in n)
    return I.Problem(name=name, bc=bc, n=tuple(n), length=length, a=a, c=c, nonlin="none", dt=dt,
                     Nt=Nt if Nt is not None else order + 9, alpha=alpha, order=order, complex_state=True)


# Sizes span several time-kernel tiles and ragged tails; Dirichlet sizes with
# n + 1 a power of two take the FFT-based sine transform, the others the dense one.
CASES = [
    P("d1_fast_s1", "dirichlet", (63,), 1),
    P("d1_dense_s2", "dirichlet", (50,), 2, c=200j, dt=0.005),
    P("d2_fast_s2", "dirichlet", (15, 31), 2),
    P("d2_dense_s6", "dirichlet", (13, 11), 6, a=0.02 + 1j, c=0.1 + 2j, Nt=17),
    P("p1_s1", "periodic", (64,), 1, a=0.05 + 1j),
    P("p2_s2", "periodic", (16, 32), 2),
    P("p2_s6", "periodic", (32, 16), 6, a=1j, c=0.5j, Nt=17, dt=0.002),
    P("d2_bluestein_s2", "dirichlet", (9, 7), 2, Nt=30),                  # Ns = 29: Bluestein window
]
IDS = [p.name for p in CASES]


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_complex_precond_apply(expd, p):
    r = cfield((p.Ns,) + p.n, 1)
    ref = O.precond_apply(O.spec_of(p), r)
    S = torch.empty_like(dev(r))
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.precond_apply(dev(r), S)
    assert relmax(host(S), ref) < 1e-11


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_complex_residual(expd, p):
    sp = O.spec_of(p)
    u0 = cfield(p.n, 2)
    f = cfield((p.Nt,) + p.n, 3)
    U = cfield((p.Nt,) + p.n, 4)
    Us = np.concatenate([u0[None], U[: p.order - 1]])
    ref = O.residual(sp, U[p.order - 1:], O.rhs_known(sp, Us, f))
    R = torch.empty((p.Ns,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, startup=expd.STARTUP_GIVEN)) as plan:
        plan.residual(dev(u0), dev(f), dev(U), R)
    assert relmax(host(R), ref) < 1e-11


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_complex_solvers_match_sequential(expd, p):
    sp = O.spec_of(p)
    u0 = cfield(p.n, 5)
    f = cfield((p.Nt,) + p.n, 6)
    seq = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=300)) as plan:
        plan.solve_sequential(dev(u0), dev(f), U)
        assert O.rel_error(host(U), seq) < 1e-12
        for fn in (plan.solve_gmres, plan.solve_fp):
            U.zero_()
            fn(dev(u0), dev(f), U)
            assert O.rel_error(host(U), seq) < 1e-10, fn.__name__


@pytest.mark.parametrize("p", CASES[:4], ids=IDS[:4])
def test_complex_gmres_history_matches_oracle(expd, p):
    sp = O.spec_of(p.with_(alpha=0.3))            # slower convergence: a longer history
    u0 = cfield(p.n, 7)
    f = cfield((p.Nt,) + p.n, 8)
    ref = O.gmres(sp, u0, f, tol=1e-12, restart=20)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p.with_(alpha=0.3), tol=1e-12, max_iter=200)) as plan:
        info = plan.solve_gmres(dev(u0), dev(f), U)
    h_gpu = np.array(info["history"])
    k = min(len(h_gpu), len(ref.history))
    big = np.array(ref.history[:k]) > 1e-9
    assert k > 2
    assert np.allclose(h_gpu[:k][big], np.array(ref.history[:k])[big], rtol=1e-6)


@pytest.mark.parametrize("Nt", (50, 200))
def test_schrodinger_1d_one_gmres_iteration(expd, Nt):
    # Sec. 7: one GMRES iteration on the 1D Schrodinger problem (h = 1/128,
    # dt = 0.01, alpha_opt, u_0 = sin(pi x)), to the paper's 1e-10 error
    p = I.SCHRODINGER_1D.with_(Nt=Nt)
    u0, f = I.make_inputs(p)
    seq = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, max_iter=50)) as plan:
        info = plan.solve_gmres(dev(u0), None, U)
    assert info["iterations"] == 1
    assert O.rel_error(host(U), seq) < 1e-10


@pytest.mark.parametrize("Nt", (20, 80))
def test_schrodinger_2d_three_gmres_iterations(expd, Nt):
    # Sec. 7: three GMRES iterations on the 2D BDF2 Schrodinger problem
    # (h = 1/40, dt = 0.05, c = 200i, the Gaussian wave packet)
    p = I.SCHRODINGER_2D.with_(Nt=Nt)
    u0, f = I.make_inputs(p)
    seq = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, max_iter=50)) as plan:
        info = plan.solve_gmres(dev(u0), None, U)
    assert info["iterations"] == 3
    assert O.rel_error(host(U), seq) < 1e-10


def test_complex_host_pointers(expd):
    p = CASES[2]
    sp = O.spec_of(p)
    u0 = cfield(p.n, 9)
    f = cfield((p.Nt,) + p.n, 10)
    seq = O.sequential_solve(sp, u0, f)[1:]
    U = np.zeros((p.Nt,) + p.n, dtype=np.complex128)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=300)) as plan:
        plan.solve_gmres(np.ascontiguousarray(u0), np.ascontiguousarray(f), U)
    assert O.rel_error(U, seq) < 1e-10


def test_complex_state_rejects_real_arrays_and_bicgstab(expd):
    p = CASES[0]
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with pytest.raises(ValueError):
            plan.solve_gmres(U[0], None, U)
        Uc = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
        with pytest.raises(expd.ExpdError) as ei:
            plan.solve_bicgstab(dev(cfield(p.n, 1)), None, Uc)
        assert ei.value.status == expd.ERR_UNSUPPORTED


@pytest.mark.parametrize("p", [CASES[0], CASES[3], CASES[5]], ids=[IDS[0], IDS[3], IDS[5]])
def test_complex_footprint_matches_allocation(expd, p):
    # expd_plan_footprint_bytes predicts what a complex-state plan allocates
    spec = expd.spec_from_problem(p, max_iter=20)
    with expd.plan_create(spec) as plan:
        assert plan.workspace_bytes() == expd.plan_footprint_bytes(spec)
        U = torch.empty((p.Nt,) + p.n, dtype=torch.complex128, device=DEV)
        plan.solve_gmres(dev(cfield(p.n, 1)), dev(cfield((p.Nt,) + p.n, 2)), U, allow_not_converged=True)
        flags = expd.FOOTPRINT_SOURCE | expd.FOOTPRINT_GMRES
        assert plan.workspace_bytes() == expd.plan_footprint_bytes(spec, flags)
