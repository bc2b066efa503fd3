"""CUDA path vs the CPU oracle, through the C ABI (marked gpu).

Tolerances: the float64 path must match the oracle to 1e-11 relative (the
stated 1e-10 bar with margin) on every element; float32-preconditioner (mixed)
operations that are not refined are held to the float32 bound eps32/alpha
(float32 rounding in the scaled time DFT, amplified at most 1/alpha by the
Gamma_alpha^-1 scaling of Eq. (3.3)); solves of either precision must meet the
workload's tolerance in the L^inf(0,T;L^2) relative error of Sec. 7.
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
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def slice_relmax(U, ref):
    """Element-wise error of every time slice relative to that slice's own
    largest value, maximised over the slices: no single grid point of any
    slice may be off by more than the bar it is held to.

    A solve stopped at the workload's tolerance targets Sec. 7's norm
    max_n ||e_n||_2 / max_n ||u_n||_2; a grid-point error spread like noise
    over the slice exceeds its slice's L2 ratio by the field's peak-to-RMS
    factor (measured up to about 4 on the Allen-Cahn fields), so at the
    workload tolerance the element-wise bar is ELEMENTWISE_FACTOR * tol.  Runs
    at the float64 parity bar (solver tol 1e-12 or below) are held to 1e-10
    element-wise as well."""
    d = np.abs(U - ref).reshape(U.shape[0], -1).max(axis=1)
    r = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return float((d / np.maximum(r, 1e-300)).max())


ELEMENTWISE_FACTOR = 10.0


def elementwise_bar(tight, tol):
    return 1e-10 if tight else ELEMENTWISE_FACTOR * tol


def P(name, bc, n, order, nonlin="none", Nt=None, alpha=1e-2, a=None, c=0.1, dt=0.01, forcing=False, b=()):
    length = tuple(2 * math.pi if bc == "periodic" else 1.0 for _ in n)
    if a is None:
        a = 0.05 if bc == "periodic" else 0.01
    return I.Problem(name=name, bc=bc, n=tuple(n), length=length, a=a, c=c, nonlin=nonlin, dt=dt,
                     Nt=Nt if Nt is not None else order + 9, alpha=alpha, order=order, forcing=forcing, b=tuple(b))


# Sizes span several time-kernel tiles (8 modes each) and ragged tails:
# periodic 1D n=64 -> 33 modes, 2D 16x32 -> 16*17 = 272 modes, Dirichlet 13x11 -> 143.
# Dirichlet sizes with n + 1 a power of two take the FFT-based sine transforms.
CASES = [
    P("p1d_s1", "periodic", (64,), 1),
    P("p1d_s2_np2", "periodic", (64,), 2, Nt=12),          # Ns = 11 (Bluestein)
    P("p2d_s1", "periodic", (16, 32), 1, Nt=16),           # Ns = 16 (radix-2)
    P("p2d_s6", "periodic", (16, 32), 6, Nt=20),           # Ns = 15 (Bluestein)
    P("p2d_s3", "periodic", (32, 16), 3, Nt=10),           # Ns = 8
    P("d1d_s1", "dirichlet", (37,), 1, Nt=9),
    P("d2d_s2", "dirichlet", (13, 11), 2, Nt=12),
    P("d2d_s6", "dirichlet", (13, 11), 6, Nt=14),
    P("p2d_ac_s1", "periodic", (16, 32), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=16, alpha=1e-3),
    P("p2d_ac_s2", "periodic", (16, 16), 2, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=21, alpha=1e-3),
    P("d2d_ac_s2", "dirichlet", (9, 12), 2, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=12, alpha=1e-3),
    # n + 1 a power of two: FFT-based sine transforms instead of the dense ones
    P("d1d_fast_s2", "dirichlet", (63,), 2, Nt=12),
    P("d2d_fast_s6", "dirichlet", (15, 31), 6, Nt=14),
    P("d2d_fast_ac_s1", "dirichlet", (31, 15), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=16, alpha=1e-3),
]
IDS = [p.name for p in CASES]


def rand_field(p, lead, seed, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal(tuple(lead) + p.n)


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_precond_apply_fp64(expd, p):
    r = rand_field(p, (p.Ns,), 1)
    ref = O.precond_apply(O.spec_of(p), r)
    S = torch.empty_like(dev(r))
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.precond_apply(dev(r), S)
    assert relmax(host(S), ref) < 1e-11


@pytest.mark.parametrize("p", CASES[:5], ids=IDS[:5])
def test_precond_apply_mixed_is_float32_accurate(expd, p):
    # float32 steps (a)-(c): error bound ~ eps32 * log2(L) / alpha relative
    r = rand_field(p, (p.Ns,), 2)
    ref = O.precond_apply(O.spec_of(p), r)
    S = torch.empty_like(dev(r))
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED)) as plan:
        plan.precond_apply(dev(r), S)
    bound = 6e-8 * 16 / p.alpha
    assert relmax(host(S), ref) < bound


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_residual_fp64(expd, p):
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


@pytest.mark.parametrize("p", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_fp_matches_sequential(expd, p, prec):
    sp = O.spec_of(p)
    rng = np.random.default_rng(4)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=200)) as plan:
        info = plan.solve_fp(dev(u0), None if f is None else dev(f), U)
    assert O.rel_error(host(U), ref) < 1e-10, info


GUESSES = ["linear", "zero"]


def guess_code(expd, guess):
    return expd.GUESS_LINEAR if guess == "linear" else expd.GUESS_ZERO


@pytest.mark.parametrize("guess", GUESSES)
@pytest.mark.parametrize("p", [CASES[i] for i in (0, 3, 6, 8, 9)], ids=[IDS[i] for i in (0, 3, 6, 8, 9)])
def test_richardson_iterates_match_oracle(expd, p, guess):
    # per-iteration parity: the k-th iterate of the GPU fixed point equals the
    # oracle's, from either initial iterate
    sp = O.spec_of(p)
    rng = np.random.default_rng(5)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    for k in (1, 2, 3):
        ref = O.richardson(sp, u0, None, max_iter=k, init=guess).U[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        spec = expd.spec_from_problem(p, tol=1e-300, max_iter=k, guess=guess_code(expd, guess))
        with expd.plan_create(spec) as plan:
            info = plan.solve_fp(dev(u0), None, U, allow_not_converged=True)
        assert info["iterations"] == k
        assert O.rel_error(host(U), ref) < 1e-12


@pytest.mark.parametrize("p", [c for c in CASES if c.nonlin == "none"], ids=[c.name for c in CASES if c.nonlin == "none"])
def test_gmres_matches_oracle(expd, p):
    sp = O.spec_of(p)
    rng = np.random.default_rng(6)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    pr = p.with_(alpha=0.3)       # slower convergence -> a longer history to compare
    spr = O.spec_of(pr)
    ref = O.gmres(spr, u0, f, tol=1e-12, restart=20)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(pr, tol=1e-12, max_iter=200)) as plan:
        info = plan.solve_gmres(dev(u0), dev(f), U)
    seq = O.sequential_solve(spr, u0, f)[1:]
    assert O.rel_error(host(U), seq) < 1e-10
    h_gpu = np.array(info["history"][: len(ref.history)])
    h_ref = np.array(ref.history[: len(h_gpu)])
    k = min(len(h_gpu), len(h_ref))
    big = h_ref[:k] > 1e-9
    assert np.allclose(h_gpu[:k][big], h_ref[:k][big], rtol=1e-6)


def test_startup_given_and_host_pointers(expd):
    p = P("p2d_s3", "periodic", (16, 16), 3, Nt=12)
    sp = O.spec_of(p)
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal(p.n)
    Ustart = np.concatenate([u0[None], rng.standard_normal((2,) + p.n)])
    ref = O.sequential_solve(sp, u0, None, U_start=Ustart)[1:]
    Uh = np.zeros((p.Nt,) + p.n)
    Uh[:2] = Ustart[1:]
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-13, startup=expd.STARTUP_GIVEN)) as plan:
        plan.solve_fp(u0, None, Uh)                      # host numpy buffers
        Ud = dev(Uh)
        Ud[2:] = 0
        plan.solve_fp(dev(u0), None, Ud)                 # device buffers
    assert O.rel_error(Uh, ref) < 1e-11
    assert np.array_equal(host(Ud), Uh)


def test_deterministic_repeat(expd):
    p = CASES[9]
    u0 = np.random.default_rng(8).uniform(-0.9, 0.9, p.n)
    outs = []
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED)) as plan:
        for _ in range(2):
            U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
            plan.solve_fp(dev(u0), None, U)
            outs.append(host(U))
    assert np.array_equal(outs[0], outs[1])


def test_not_converged_and_diverged_status(expd):
    p = CASES[8]
    u0 = np.random.default_rng(9).uniform(-0.9, 0.9, p.n)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-15, max_iter=1)) as plan:
        with pytest.raises(expd.ExpdError) as ei:
            plan.solve_fp(dev(u0), None, U)
        assert ei.value.status == expd.ERR_NOT_CONVERGED
        bad = u0.copy()
        bad[0, 0] = np.nan
        with pytest.raises(expd.ExpdError) as ei:
            plan.solve_fp(dev(bad), None, U)
        assert ei.value.status == expd.ERR_DIVERGED


def test_minimum_window_and_large_alpha(expd):
    # Ns = 2 (Nt = s + 1) with alpha = 0.4: the iteration matrix's spectral radius
    # is about alpha/(1 - alpha) = 0.67 (Theorem 3.1 / 4.1), slow but convergent
    for order in (1, 2, 6):
        p = P(f"min_s{order}", "periodic", (16,), order, Nt=order + 1, alpha=0.4)
        sp = O.spec_of(p)
        u0 = np.random.default_rng(order).standard_normal(p.n)
        ref = O.sequential_solve(sp, u0)[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, tol=1e-13, max_iter=400)) as plan:
            plan.solve_fp(dev(u0), None, U)
        assert O.rel_error(host(U), ref) < 1e-10


def test_alpha_beyond_convergence_bound_reports_divergence(expd):
    # alpha = 0.9 with E ~ 1: spectral radius alpha/(1 - alpha) = 9 > 1.  From
    # the zero iterate (the linear guess is already this homogeneous problem's
    # solution, so it would stop at once)
    p = P("div", "periodic", (16,), 1, Nt=4, alpha=0.9, a=1e-4, c=0.0)
    u0 = np.random.default_rng(0).standard_normal(p.n)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    spec = expd.spec_from_problem(p, tol=1e-13, max_iter=400, guess=expd.GUESS_ZERO)
    with expd.plan_create(spec) as plan:
        with pytest.raises(expd.ExpdError) as ei:
            info = plan.solve_fp(dev(u0), None, U)
        assert ei.value.status == expd.ERR_DIVERGED


# ---------------------------------------------------------------- full size --
def solve_full(expd, p, precision, solver=None, tol=None):
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, max_iter=200, tol=tol)) as plan:
        fn = plan.solve_gmres if (solver or p.solver) == "gmres" else plan.solve_fp
        info = fn(dev(u0), None if f is None else dev(f), U)
    return u0, f, host(U), info


_REF = {}


def sequential_ref(p, u0, f):
    """The oracle's sequential solution of a full-size workload, computed once per module."""
    if p.name not in _REF:
        _REF[p.name] = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    return _REF[p.name]


def test_heat1d_full_exact_solution(expd):
    p = I.HEAT1D
    u0, f, U8, info8 = solve_full(expd, p, expd.PREC_FP64)          # the workload's tol 1e-8
    u0, f, U, info = solve_full(expd, p, expd.PREC_FP64, tol=1e-13)  # float64 parity bar
    x = I.grid_coords(p)[0]
    rng = np.random.default_rng(p.seed)
    ak, bk = rng.standard_normal(16), rng.standard_normal(16)
    exact = np.array([sum(math.exp(-k * k * (n + 1) * p.dt) * (ak[k - 1] * np.cos(k * x) + bk[k - 1] * np.sin(k * x))
                          / k**2 for k in range(1, 17)) for n in range(p.Nt)])
    assert O.rel_error(U8, exact) < p.tol
    assert O.rel_error(U, exact) < 1e-10
    seq = O.sequential_solve(O.spec_of(p), u0)[1:]
    assert O.rel_error(U, seq) < 1e-10
    assert slice_relmax(U, seq) < 1e-10
    assert slice_relmax(U8, seq) < elementwise_bar(False, p.tol)
    assert info["iterations"] <= 8


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tight"])
def test_allen_cahn_256_full(expd, prec):
    p = I.ALLEN_CAHN_256
    tight = prec == "fp64_tight"
    u0, f, U, info = solve_full(expd, p, expd.PREC_MIXED if prec == "mixed" else expd.PREC_FP64,
                                tol=1e-13 if tight else None)
    ref = sequential_ref(p, u0, None)
    bar = 1e-10 if tight else p.tol
    assert O.rel_error(U, ref) < bar, info
    assert slice_relmax(U, ref) < elementwise_bar(tight, p.tol), info


# The 512^2 x 256 order-6 Allen-Cahn workload: its tolerance 1e-8 on both
# paths, and the float64 path held to the 1e-10 parity bar at solver tol 1e-12.
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tight"])
def test_allen_cahn_512_order6_full(expd, prec):
    p = I.ALLEN_CAHN_512_S6
    tight = prec == "fp64_tight"
    u0, f, U, info = solve_full(expd, p, expd.PREC_MIXED if prec == "mixed" else expd.PREC_FP64,
                                tol=1e-12 if tight else None)
    ref = sequential_ref(p, u0, None)
    bar = 1e-10 if tight else p.tol
    assert O.rel_error(U, ref) < bar, info
    assert slice_relmax(U, ref) < elementwise_bar(tight, p.tol), info


# The 1024^2 x 128 Dirichlet heat workload (s = 2, GMRES or BiCGStab, tol 1e-9):
# the float64 path (float64 dense sine products and preconditioner) at the
# workload's tolerance and at the 1e-10 parity bar (solver tol 1e-12), and the
# mixed path (tensor-core sine transforms, float32 preconditioner inside
# float64 residual refinement) at the workload's tolerance.
@pytest.mark.parametrize("case", ["fp64_gmres", "fp64_tight_gmres", "mixed_gmres", "mixed_bicgstab"])
def test_heat_dirichlet_1024_full(expd, case):
    p = I.HEAT_DIRICHLET_1024
    tight = "tight" in case
    prec = expd.PREC_MIXED if case.startswith("mixed") else expd.PREC_FP64
    solver = "bicgstab" if case.endswith("bicgstab") else "gmres"
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=prec, max_iter=200,
                                                 tol=1e-12 if tight else None)) as plan:
        fn = plan.solve_bicgstab if solver == "bicgstab" else plan.solve_gmres
        info = fn(dev(u0), dev(f), U)
    Uh = host(U)
    ref = sequential_ref(p, u0, f)
    bar = 1e-10 if tight else p.tol
    assert O.rel_error(Uh, ref) < bar, info
    assert slice_relmax(Uh, ref) < elementwise_bar(tight, p.tol), info
    if prec == expd.PREC_MIXED:
        assert info["refinements"] >= 1, info


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
@pytest.mark.parametrize("p", [c for c in CASES if c.nonlin == "none"], ids=[c.name for c in CASES if c.nonlin == "none"])
def test_mixed_krylov_refinement_reaches_float64_accuracy(expd, p, solver):
    # the float32 preconditioner's rounding (about eps32/alpha) limits only how
    # fast the refinement restarts contract: the solution reaches the float64
    # parity bar against sequential stepping
    sp = O.spec_of(p)
    rng = np.random.default_rng(14)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=400)) as plan:
        fn = plan.solve_bicgstab if solver == "bicgstab" else plan.solve_gmres
        info = fn(dev(u0), dev(f), U)
    Uh = host(U)
    assert O.rel_error(Uh, ref) < 1e-10, info
    assert slice_relmax(Uh, ref) < 1e-10, info
    assert info["refinements"] >= 1, info
    assert info["final_measure"] <= 1e-12 / math.sqrt(p.Ns), info


def test_info_phase_times(expd):
    p = CASES[6]
    rng = np.random.default_rng(15)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-12)) as plan:
        for fn in (plan.solve_fp, plan.solve_gmres, plan.solve_bicgstab):
            info = fn(dev(u0), dev(f), U)
            assert info["ms_setup"] > 0 and info["ms_iterate"] > 0 and info["ms_output"] > 0, info


def test_time_limit_and_cancel_status(expd):
    # a time limit that has run out stops the solve between iterations with
    # EXPD_ERR_TIMEOUT; expd_plan_cancel stops the next solve with
    # EXPD_ERR_CANCELLED (the request is consumed: the solve after it succeeds)
    p = CASES[0].with_(alpha=0.3)
    rng = np.random.default_rng(16)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    ref = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-13, max_iter=400, time_limit_ms=1e-6)) as plan:
        for fn in (plan.solve_fp, plan.solve_gmres, plan.solve_bicgstab):
            with pytest.raises(expd.ExpdError) as ei:
                fn(dev(u0), dev(f), U)
            assert ei.value.status == expd.ERR_TIMEOUT
    with expd.plan_create(expd.spec_from_problem(p, tol=1e-13, max_iter=400)) as plan:
        for fn in (plan.solve_fp, plan.solve_gmres, plan.solve_bicgstab):
            plan.cancel()
            with pytest.raises(expd.ExpdError) as ei:
                fn(dev(u0), dev(f), U)
            assert ei.value.status == expd.ERR_CANCELLED
            fn(dev(u0), dev(f), U)
            assert O.rel_error(host(U), ref) < 1e-10


def test_footprint_matches_allocation(expd):
    # expd_plan_footprint_bytes predicts exactly what a plan allocates (admission control)
    cases = [(CASES[0], expd.PREC_FP64, 0), (CASES[3], expd.PREC_MIXED, 0), (CASES[6], expd.PREC_MIXED, 0),
             (CASES[9], expd.PREC_MIXED, 0), (CASES[10], expd.PREC_FP64, 0)]
    for p, prec, _ in cases:
        spec = expd.spec_from_problem(p, precision=prec)
        want = expd.plan_footprint_bytes(spec)
        with expd.plan_create(spec) as plan:
            assert plan.workspace_bytes() == want, p.name
            if p.nonlin == "none":
                u0 = np.zeros(p.n)
                f = np.zeros((p.Nt,) + p.n)
                U = np.zeros((p.Nt,) + p.n)
                plan.solve_gmres(u0, f, U)          # host pointers, a source, GMRES
                flags = expd.FOOTPRINT_SOURCE | expd.FOOTPRINT_HOST | expd.FOOTPRINT_GMRES
                assert plan.workspace_bytes() == expd.plan_footprint_bytes(spec, flags), p.name


# ------------------------------------------- register-resident time kernel --
# Power-of-two windows Ns in {16, 32, 64} with the float32 preconditioner run a
# kernel that keeps each mode's time column in registers; EXPD_TIME_KERNEL=smem
# selects the shared-memory kernel instead.  Grids give a ragged last CTA of
# 128 columns: periodic 16x64 -> 16*33 = 528 columns, Dirichlet 13x23 -> 299.
REG_CASES = [
    P(f"reg_{bc[0]}_ns{ns}_s{s}", bc, (16, 64) if bc == "periodic" else (13, 23), s, Nt=ns + s - 1,
      nonlin=nl, a=0.01, c=0.0 if nl != "none" else 0.1, dt=1e-3, alpha=1e-3)
    for ns in (16, 32, 64) for bc in ("periodic", "dirichlet") for (s, nl) in ((1, "allen_cahn"), (2, "none"), (6, "none"))
]
REG_IDS = [p.name for p in REG_CASES]


def _with_kernel(monkeypatch, kind):
    if kind == "smem":
        monkeypatch.setenv("EXPD_TIME_KERNEL", "smem")
    else:
        monkeypatch.delenv("EXPD_TIME_KERNEL", raising=False)


@pytest.mark.parametrize("p", REG_CASES, ids=REG_IDS)
def test_register_time_kernel_precond(expd, p, monkeypatch):
    r = rand_field(p, (p.Ns,), 11)
    ref = O.precond_apply(O.spec_of(p), r)
    out = {}
    for kind in ("reg", "smem"):
        _with_kernel(monkeypatch, kind)
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED)) as plan:
            plan.precond_apply(dev(r), S)
        out[kind] = host(S)
    bound = 6e-8 * 16 / p.alpha
    assert relmax(out["reg"], ref) < bound
    assert relmax(out["smem"], ref) < bound
    assert relmax(out["reg"], out["smem"]) < bound


@pytest.mark.parametrize("p", REG_CASES, ids=REG_IDS)
def test_register_time_kernel_solve(expd, p, monkeypatch):
    # the mixed solve runs the register kernel for its float32 sweeps (and for
    # accurate sweeps stored in float64); the per-slice norms its
    # transpose-reduce produces drive the stopping test, so the first measures
    # of the two kernels must agree
    sp = O.spec_of(p)
    rng = np.random.default_rng(12)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    ref = O.sequential_solve(sp, u0, f)[1:]
    res = {}
    for kind in ("reg", "smem"):
        _with_kernel(monkeypatch, kind)
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=200)) as plan:
            info = plan.solve_fp(dev(u0), None if f is None else dev(f), U)
        assert O.rel_error(host(U), ref) < 1e-10, (kind, info)
        res[kind] = info
    # the first sweep's measure is far above float32 rounding; later float32
    # sweeps reach their rounding floor, where the two kernels' noise differs
    h_reg = np.array(res["reg"]["history"][:2])
    h_smem = np.array(res["smem"]["history"][:2])
    assert np.allclose(h_reg, h_smem, rtol=1e-3), (h_reg, h_smem)
    assert abs(res["reg"]["fp32_iterations"] - res["smem"]["fp32_iterations"]) <= 1


# ------------------------------------------------- sequential time stepping --
@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_sequential_stepper_matches_oracle(expd, p):
    # the GPU stepper is the exact solution of the all-at-once system (block
    # lower-triangular), so it matches the oracle's stepping to float64 rounding
    sp = O.spec_of(p)
    rng = np.random.default_rng(13)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.solve_sequential(dev(u0), None if f is None else dev(f), U)
    assert O.rel_error(host(U), ref) < 1e-12


def test_sequential_stepper_full_size_allen_cahn_256(expd):
    p = I.ALLEN_CAHN_256
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.solve_sequential(dev(u0), None, U)
    Uh = host(U)
    sp = O.spec_of(p)
    # every slice against the oracle's stepping (a few seconds on the CPU at this size)
    ref = O.sequential_solve(sp, u0, None)[1:]
    assert O.rel_error(Uh, ref) < 1e-12


def test_fast_sine_transform_full_size_gmres(expd):
    # heat equation on (0,1)^2 with 1023^2 interior points (h = 1/1024): the
    # FFT-based sine transforms at full size, GMRES as for the 1024^2 workload
    p = I.HEAT_DIRICHLET_1024.with_(name="heat_dirichlet_1023", n=(1023, 1023), Nt=32)
    u0, f, U, info = solve_full(expd, p, expd.PREC_FP64)
    ref = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    assert O.rel_error(U, ref) < 1e-8, info
    Useq = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.solve_sequential(dev(u0), dev(f), Useq)
    assert O.rel_error(host(Useq), ref) < 1e-12


# ------------------------------------------------------------------ BiCGStab --
@pytest.mark.parametrize("p", [c for c in CASES if c.nonlin == "none"], ids=[c.name for c in CASES if c.nonlin == "none"])
def test_bicgstab_matches_oracle(expd, p):
    sp = O.spec_of(p)
    rng = np.random.default_rng(14)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    pr = p.with_(alpha=0.3)       # slower convergence -> a longer history to compare
    spr = O.spec_of(pr)
    ref = O.bicgstab(spr, u0, f, tol=1e-12 / math.sqrt(pr.Ns))
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(pr, tol=1e-12, max_iter=200)) as plan:
        info = plan.solve_bicgstab(dev(u0), dev(f), U)
    seq = O.sequential_solve(spr, u0, f)[1:]
    assert O.rel_error(host(U), seq) < 1e-10
    assert O.rel_error(ref.U[1:], seq) < 1e-10
    # iterate-by-iterate parity: the relative preconditioned residuals agree
    h_gpu = np.array(info["history"])
    h_ref = np.array(ref.history)
    k = min(len(h_gpu), len(h_ref))
    big = h_ref[:k] > 1e-8
    assert np.allclose(h_gpu[:k][big], h_ref[:k][big], rtol=1e-6), (h_gpu[:k], h_ref[:k])


def test_bicgstab_full_size_heat_dirichlet(expd):
    p = I.HEAT_DIRICHLET_1024.with_(name="heat_dirichlet_1023_bicgstab", n=(1023, 1023), Nt=32)
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, max_iter=200)) as plan:
        info = plan.solve_bicgstab(dev(u0), dev(f), U)
    ref = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    assert O.rel_error(host(U), ref) < 1e-8, info


# ------------------------------------- radix-4 shared-memory row / column FFTs --
@pytest.mark.parametrize("p", [CASES[i] for i in (2, 3, 8, 9)], ids=[IDS[i] for i in (2, 3, 8, 9)])
def test_radix4_fft_path(expd, p, monkeypatch):
    # EXPD_FFT_KERNEL=radix4 keeps the shared-memory row and column FFTs (used
    # for sizes and precisions the four-step kernels do not take) covered
    monkeypatch.setenv("EXPD_FFT_KERNEL", "radix4")
    sp = O.spec_of(p)
    r = rand_field(p, (p.Ns,), 15)
    S = torch.empty_like(dev(r))
    rng = np.random.default_rng(16)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=200)) as plan:
        plan.precond_apply(dev(r), S)
        plan.solve_fp(dev(u0), None if f is None else dev(f), U)
    assert relmax(host(S), O.precond_apply(sp, r)) < 6e-8 * 16 / p.alpha
    assert O.rel_error(host(U), O.sequential_solve(sp, u0, f)[1:]) < 1e-10


# --------------------------------------- inexact Newton, mean Jacobian at u0 --
NL_CASES = [c for c in CASES if c.nonlin != "none"]
NL_IDS = [c.name for c in NL_CASES]


@pytest.mark.parametrize("guess", GUESSES)
@pytest.mark.parametrize("p", NL_CASES, ids=NL_IDS)
def test_mean_jacobian_iterates_match_oracle(expd, p, guess):
    sp = O.spec_of(p)
    u0 = np.random.default_rng(17).uniform(-0.8, 0.8, p.n)
    for k in (1, 2, 3):
        ref = O.richardson(sp, u0, None, max_iter=k, jacobian="mean_u0", init=guess).U[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        spec = expd.spec_from_problem(p, tol=1e-300, max_iter=k, jacobian=expd.JAC_MEAN_U0,
                                      guess=guess_code(expd, guess))
        with expd.plan_create(spec) as plan:
            info = plan.solve_fp(dev(u0), None, U, allow_not_converged=True)
        assert info["iterations"] == k
        assert O.rel_error(host(U), ref) < 1e-12


@pytest.mark.parametrize("p", NL_CASES, ids=NL_IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mean_jacobian_solve_matches_sequential(expd, p, prec):
    sp = O.spec_of(p)
    u0 = np.random.default_rng(18).uniform(-0.8, 0.8, p.n)
    ref = O.sequential_solve(sp, u0)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    spec = expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=200, jacobian=expd.JAC_MEAN_U0)
    with expd.plan_create(spec) as plan:
        info = plan.solve_fp(dev(u0), None, U)
    assert O.rel_error(host(U), ref) < 1e-10, info


def test_mean_jacobian_full_size_allen_cahn_256(expd):
    p = I.ALLEN_CAHN_256
    u0, _ = I.make_inputs(p)
    ref = O.sequential_solve(O.spec_of(p), u0)[1:]
    its = {}
    for jac in (expd.JAC_LAGGED, expd.JAC_MEAN_U0):
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, max_iter=200, jacobian=jac)
        with expd.plan_create(spec) as plan:
            info = plan.solve_fp(dev(u0), None, U)
        assert O.rel_error(host(U), ref) < p.tol, (jac, info)
        its[jac] = info["iterations"]
    assert its[expd.JAC_MEAN_U0] <= its[expd.JAC_LAGGED], its


# ------------------------------------------- advection-diffusion (periodic) --
# complex symbol -a|k|^2 - i b.k - c: register kernel (Ns = 16, 32) and
# shared-memory kernel (Ns = 11, Bluestein), float64, mixed and double-float
ADV_CASES = [
    P("adv_1d_s1", "periodic", (64,), 1, Nt=16, b=(1.5,)),
    P("adv_2d_s2", "periodic", (16, 32), 2, Nt=12, b=(0.7, -1.2)),
    P("adv_2d_s6", "periodic", (32, 32), 6, Nt=37, b=(2.0, 0.5)),
    P("adv_2d_ac_s1", "periodic", (16, 32), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=16, alpha=1e-3,
      b=(0.5, 1.0)),
]
ADV_IDS = [p.name for p in ADV_CASES]


@pytest.mark.parametrize("p", ADV_CASES, ids=ADV_IDS)
def test_advection_precond_and_residual(expd, p):
    sp = O.spec_of(p)
    r = rand_field(p, (p.Ns,), 21)
    ref = O.precond_apply(sp, r)
    for prec, bound in ((expd.PREC_FP64, 1e-11), (expd.PREC_MIXED, 6e-8 * 16 / p.alpha)):
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=prec)) as plan:
            plan.precond_apply(dev(r), S)
        assert relmax(host(S), ref) < bound, prec
    rng = np.random.default_rng(22)
    u0 = rng.uniform(-0.5, 0.5, p.n)
    U = rng.uniform(-0.5, 0.5, (p.Nt,) + p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    U_start = np.concatenate([u0[None], U[: p.order - 1]])
    ref = O.residual(sp, U[p.order - 1:], O.rhs_known(sp, U_start, f))
    R = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.residual(dev(u0), dev(f), dev(U), R)
    assert relmax(host(R), ref) < 1e-11


@pytest.mark.parametrize("p", ADV_CASES, ids=ADV_IDS)
def test_advection_solvers_match_sequential(expd, p):
    sp = O.spec_of(p)
    rng = np.random.default_rng(23)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    ref = O.sequential_solve(sp, u0, f)[1:]
    fd = None if f is None else dev(f)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.solve_sequential(dev(u0), fd, U)
        assert O.rel_error(host(U), ref) < 1e-12
    for prec in (expd.PREC_FP64, expd.PREC_MIXED):
        with expd.plan_create(expd.spec_from_problem(p, precision=prec, tol=1e-12, max_iter=200)) as plan:
            info = plan.solve_fp(dev(u0), fd, U)
        assert O.rel_error(host(U), ref) < 1e-10, (prec, info)
    if p.nonlin == "none":
        with expd.plan_create(expd.spec_from_problem(p, tol=1e-12, max_iter=200)) as plan:
            plan.solve_gmres(dev(u0), fd, U)
            assert O.rel_error(host(U), ref) < 1e-10
            plan.solve_bicgstab(dev(u0), fd, U)
            assert O.rel_error(host(U), ref) < 1e-10


@pytest.mark.parametrize("guess", GUESSES)
def test_advection_richardson_iterates_match_oracle(expd, guess):
    p = ADV_CASES[1]
    sp = O.spec_of(p)
    rng = np.random.default_rng(24)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    for k in (1, 2, 3):
        ref = O.richardson(sp, u0, f, max_iter=k, init=guess).U[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        spec = expd.spec_from_problem(p, tol=1e-300, max_iter=k, guess=guess_code(expd, guess))
        with expd.plan_create(spec) as plan:
            plan.solve_fp(dev(u0), dev(f), U, allow_not_converged=True)
        assert O.rel_error(host(U), ref) < 1e-12


# ------------------------------------------------------------ largest window --
@pytest.mark.parametrize("Nt,order", [(512, 1), (517, 6)])   # Ns = 512 (radix-2), 512 (order 6)
def test_largest_window(expd, Nt, order):
    p = P(f"max_ns_s{order}", "periodic", (16,), order, Nt=Nt, alpha=0.05, a=0.05, c=0.1, dt=1e-3, forcing=True)
    assert p.Ns == 512
    sp = O.spec_of(p)
    rng = np.random.default_rng(25)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    for prec in (expd.PREC_FP64, expd.PREC_MIXED):
        with expd.plan_create(expd.spec_from_problem(p, precision=prec, tol=1e-12, max_iter=200)) as plan:
            plan.solve_fp(dev(u0), dev(f), U)
        assert O.rel_error(host(U), ref) < 1e-10, prec


# --------------------------------------------------- sweeps as CUDA graphs --
@pytest.mark.parametrize("p", [CASES[8], CASES[9], CASES[0]], ids=[IDS[8], IDS[9], IDS[0]])
def test_graph_sweeps_match_direct_launches(expd, p):
    # on a stream of its own a solve relaunches each phase's sweep as a CUDA
    # graph (captured on the second sweep of the phase, recaptured when the
    # output buffer changes); the legacy default stream launches kernel by
    # kernel: the results must agree bit for bit, call after call
    u0 = np.random.default_rng(19).uniform(-0.8, 0.8, p.n)
    f = np.random.default_rng(20).standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    fd = None if f is None else dev(f)
    for jac in (expd.JAC_LAGGED, expd.JAC_MEAN_U0):
        spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=200, jacobian=jac)
        ref = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(spec) as plan:
            plan.solve_fp(dev(u0), fd, ref)               # default stream: no graphs
        ref = host(ref)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side), expd.plan_create(spec, side) as plan:
            for k in range(3):
                U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)   # a new buffer each call
                plan.solve_fp(dev(u0), fd, U, stream=side)
                side.synchronize()
                assert np.array_equal(U.cpu().numpy(), ref), (jac, k)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("max_iter", [200, 3])
@pytest.mark.parametrize("p", [CASES[8], CASES[10], CASES[2], CASES[13]], ids=[IDS[8], IDS[10], IDS[2], IDS[13]])
def test_device_loop_matches_host_loop(expd, p, max_iter, prec, monkeypatch):
    # with EXPD_DEVICE_LOOP=1, from its second solve a plan on a capturable
    # stream runs the fixed point as one graph whose stopping test runs on the
    # GPU (while-nodes); the iterate, the iteration counts, the error-estimate
    # history and the status must be those of the host-side loop, bit for bit
    u0 = np.random.default_rng(51).uniform(-0.8, 0.8, p.n)
    f = 0.3 * np.random.default_rng(52).standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    fd = None if f is None else dev(f)
    precision = expd.PREC_MIXED if prec == "mixed" else expd.PREC_FP64
    spec = expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=max_iter)
    side = torch.cuda.Stream()
    runs = {}
    for mode in ("host", "device"):
        monkeypatch.setenv("EXPD_DEVICE_LOOP", "1" if mode == "device" else "0")
        out = []
        with torch.cuda.stream(side), expd.plan_create(spec, side) as plan:
            for _ in range(3):
                U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
                plan.timing_read(reset=True)
                info = plan.solve_fp(dev(u0), fd, U, stream=side, allow_not_converged=True)
                side.synchronize()
                info["launches"] = plan.timing_read(reset=True)["launches"]
                out.append((U.cpu().numpy(), info))
        runs[mode] = out
    # the device loop adds its init, per-sweep control and output launches
    # (and converts the float32 iterate, which the host loop's first
    # double-float sweep reads directly on register-kernel windows)
    last_h, last_d = runs["host"][-1][1], runs["device"][-1][1]
    assert last_d["launches"] - last_h["launches"] in (last_d["iterations"] + 2, last_d["iterations"] + 3)
    for (Uh, ih), (Ud, idv) in zip(runs["host"], runs["device"]):
        assert np.array_equal(Uh, Ud)
        for k in ("iterations", "fp32_iterations", "final_measure", "contraction", "history", "status"):
            assert ih[k] == idv[k], k
    if max_iter == 3:
        assert runs["device"][-1][1]["status"] == expd.ERR_NOT_CONVERGED


@pytest.mark.parametrize("p", [CASES[8], CASES[2]], ids=[IDS[8], IDS[2]])
def test_graph_recaptured_when_forcing_changes(expd, p):
    # the time kernel reads the right-hand side only on its nonzero slices (the
    # start-up slices without a forcing term, all of them with one): a plan that
    # alternates between the two must not relaunch a sweep captured for the other
    u0 = np.random.default_rng(41).uniform(-0.8, 0.8, p.n)
    f = 0.3 * np.random.default_rng(42).standard_normal((p.Nt,) + p.n)
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-12, max_iter=200)
    refs = {}
    for key, ff in (("none", None), ("f", f)):
        ref = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(spec) as plan:
            plan.solve_fp(dev(u0), None if ff is None else dev(ff), ref)   # default stream: no graphs
        refs[key] = host(ref)
    assert relmax(refs["f"], refs["none"]) > 1e-3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side), expd.plan_create(spec, side) as plan:
        for key in ("none", "none", "none", "f", "f", "none", "f"):
            U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
            plan.solve_fp(dev(u0), None if key == "none" else dev(f), U, stream=side)
            side.synchronize()
            assert np.array_equal(U.cpu().numpy(), refs[key]), key


@pytest.mark.parametrize("p", [CASES[8], CASES[6], CASES[0]], ids=[IDS[8], IDS[6], IDS[0]])
def test_graph_sequential_stepping_matches_direct(expd, p):
    u0 = np.random.default_rng(26).uniform(-0.8, 0.8, p.n)
    f = np.random.default_rng(27).standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    fd = None if f is None else dev(f)
    spec = expd.spec_from_problem(p)
    ref = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(spec) as plan:
        plan.solve_sequential(dev(u0), fd, ref)
    ref = host(ref)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side), expd.plan_create(spec, side) as plan:
        for k in range(3):
            U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
            plan.solve_sequential(dev(u0), fd, U, stream=side)
            side.synchronize()
            assert np.array_equal(U.cpu().numpy(), ref), k


# ----------------------------------------------- real-column time kernel --
# Dirichlet grids run a real-column kernel (16 columns per CTA, two per warp,
# swizzled FFT buffers, float32 combination for operator applications on the
# mixed path); EXPD_TIME_REAL=0 selects the generic kernel.  Both compute the
# same operations: the preconditioner and the residual agree to the oracle's
# tolerance of their precision, and the Krylov solves reach the float64 bar.
REAL_CASES = [c for c in CASES if c.bc == "dirichlet"] + [
    P("d2d_blue127", "dirichlet", (19, 13), 2, Nt=128, alpha=1e-3, dt=1e-3),   # Ns = 127: Bluestein L = 256
    P("d2d_pow2_32", "dirichlet", (17, 9), 1, Nt=32),                            # Ns = 32: radix-2
    # the compile-time Bluestein lengths (the pointwise steps folded into the
    # passes): L = 64, 128, 512, odd and even log2 L; a compile-time radix-2
    # window (L = Ns = 256)
    P("d2d_blue20", "dirichlet", (9, 7), 2, Nt=21, alpha=1e-3, dt=1e-3),       # Ns = 20: L = 64
    P("d2d_blue45", "dirichlet", (7, 9), 6, Nt=50, alpha=1e-3, dt=1e-3),       # Ns = 45: L = 128
    P("d2d_blue200", "dirichlet", (5, 7), 1, Nt=200, alpha=1e-3, dt=1e-3),     # Ns = 200: L = 512
    P("d2d_pow2_256", "dirichlet", (6, 5), 2, Nt=257, alpha=1e-3, dt=1e-3),    # Ns = 256: radix-2 at L = 256
]


@pytest.mark.parametrize("p", REAL_CASES, ids=[p.name for p in REAL_CASES])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_real_time_kernel_matches_generic_and_oracle(expd, p, prec, monkeypatch):
    sp = O.spec_of(p)
    r = rand_field(p, (p.Ns,), 23)
    ref = O.precond_apply(sp, r)
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    outs = {}
    for kind in ("real", "generic"):
        if kind == "generic":
            monkeypatch.setenv("EXPD_TIME_REAL", "0")
        else:
            monkeypatch.delenv("EXPD_TIME_REAL", raising=False)
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=precision)) as plan:
            plan.precond_apply(dev(r), S)
        outs[kind] = host(S)
    bound = 1e-11 if prec == "fp64" else 6e-8 * 16 / p.alpha
    assert relmax(outs["real"], ref) < bound
    assert relmax(outs["generic"], ref) < bound
    assert relmax(outs["real"], outs["generic"]) < bound
    if p.nonlin == "none":
        rng = np.random.default_rng(24)
        u0 = rng.standard_normal(p.n)
        f = rng.standard_normal((p.Nt,) + p.n)
        seq = O.sequential_solve(sp, u0, f)[1:]
        monkeypatch.delenv("EXPD_TIME_REAL", raising=False)
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=400)) as plan:
            for fn in (plan.solve_gmres, plan.solve_bicgstab, plan.solve_fp):
                info = fn(dev(u0), dev(f), U)
                assert O.rel_error(host(U), seq) < 1e-10, (fn.__name__, info)


# ------------------------------------------------- complex-column kernel --
# Periodic grids: the fixed-length complex-column time kernel (time_cplx.cu;
# compile-time FFT lengths 64-512 here, folded Bluestein passes) against the
# generic shared-memory kernel (EXPD_TIME_CPLX=0) and the oracle, on windows
# covering every compiled length, a run-time length (L = 32) and a compiled
# radix-2 window; the mixed fixed point runs its float32 and double-float
# sweeps through it.
CPLX_CASES = [
    P("p2d_blue11", "periodic", (16, 32), 1, Nt=11, alpha=1e-3, dt=1e-3),      # Ns = 11: L = 32 (run time)
    P("p2d_blue20", "periodic", (16, 32), 2, Nt=21, alpha=1e-3, dt=1e-3),      # L = 64
    P("p2d_blue45", "periodic", (16, 16), 6, Nt=50, alpha=1e-3, dt=1e-3),      # L = 128
    P("p2d_blue127", "periodic", (8, 16), 2, Nt=128, alpha=1e-3, dt=1e-3),     # L = 256
    P("p2d_blue251", "periodic", (8, 8), 6, Nt=256, alpha=1e-3, dt=1e-3),      # L = 512
    P("p2d_pow2_128", "periodic", (16, 8), 1, Nt=128, alpha=1e-3, dt=1e-3),    # radix-2, L = 128
    P("p2d_ac_blue63", "periodic", (16, 16), 2, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=64,
      alpha=1e-3),                                                              # Allen-Cahn, L = 128
]


@pytest.mark.parametrize("p", CPLX_CASES, ids=[p.name for p in CPLX_CASES])
def test_complex_column_kernel_matches_generic_and_oracle(expd, p, monkeypatch):
    sp = O.spec_of(p)
    r = rand_field(p, (p.Ns,), 27)
    ref = O.precond_apply(sp, r)
    outs = {}
    for kind in ("fixed", "generic"):
        if kind == "generic":
            monkeypatch.setenv("EXPD_TIME_CPLX", "0")
        else:
            monkeypatch.delenv("EXPD_TIME_CPLX", raising=False)
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p)) as plan:
            plan.precond_apply(dev(r), S)
        outs[kind] = host(S)
    assert relmax(outs["fixed"], ref) < 1e-11
    assert relmax(outs["generic"], ref) < 1e-11
    monkeypatch.delenv("EXPD_TIME_CPLX", raising=False)
    rng = np.random.default_rng(28)
    amp = 0.8 if p.nonlin != "none" else 1.0
    u0 = amp * rng.uniform(-1, 1, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    seq = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    for prec in (expd.PREC_FP64, expd.PREC_MIXED):
        with expd.plan_create(expd.spec_from_problem(p, precision=prec, tol=1e-12, max_iter=400)) as plan:
            fns = (plan.solve_fp,) if p.nonlin != "none" else (plan.solve_fp, plan.solve_gmres)
            for fn in fns:
                fn(dev(u0), None if f is None else dev(f), U)
                assert O.rel_error(host(U), seq) < 1e-10, (fn.__name__, prec)


# ------------------------------------------------------------------- ETD1 --
# u_n = A u_{n-1} + dt phi_1(dt L) N(u_{n-1}) (nl_form = EXPD_NLF_ETD1): the
# phi_1 tables, the one-slice shift of the transformed N, the phi_1 N(u_0)
# term of the right-hand side and the ETD sequential step, against the oracle.
ETD_CASES = [
    P("etd_p2d_ns16", "periodic", (16, 32), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=16,
      alpha=1e-3).with_(nl_form="etd1"),                                      # register kernel (mixed)
    P("etd_p2d_ns20", "periodic", (32, 16), 1, nonlin="allen_cahn", a=0.01, c=0.1, dt=2e-3, Nt=20,
      alpha=1e-3).with_(nl_form="etd1"),                                      # Bluestein window
    P("etd_d2d", "dirichlet", (9, 12), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=12,
      alpha=1e-3).with_(nl_form="etd1"),
    P("etd_p1d", "periodic", (64,), 1, nonlin="allen_cahn", a=0.05, c=0.0, dt=5e-3, Nt=24,
      alpha=1e-2).with_(nl_form="etd1"),
]
ETD_IDS = [p.name for p in ETD_CASES]


@pytest.mark.parametrize("guess", GUESSES)
@pytest.mark.parametrize("p", ETD_CASES, ids=ETD_IDS)
def test_etd1_richardson_iterates_match_oracle(expd, p, guess):
    sp = O.spec_of(p)
    assert sp.nl_form == "etd1"
    u0 = np.random.default_rng(31).uniform(-0.8, 0.8, p.n)
    for k in (1, 2, 3):
        ref = O.richardson(sp, u0, None, max_iter=k, init=guess).U[1:]
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        spec = expd.spec_from_problem(p, tol=1e-300, max_iter=k, guess=guess_code(expd, guess))
        assert spec.nl_form == expd.NLF_ETD1
        with expd.plan_create(spec) as plan:
            info = plan.solve_fp(dev(u0), None, U, allow_not_converged=True)
        assert info["iterations"] == k
        assert O.rel_error(host(U), ref) < 1e-12, (k, guess)


@pytest.mark.parametrize("p", ETD_CASES, ids=ETD_IDS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_etd1_solve_and_stepper_match_sequential(expd, p, prec):
    sp = O.spec_of(p)
    u0 = np.random.default_rng(32).uniform(-0.8, 0.8, p.n)
    ref = O.sequential_solve(sp, u0)[1:]
    precision = expd.PREC_FP64 if prec == "fp64" else expd.PREC_MIXED
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=precision, tol=1e-12, max_iter=200)) as plan:
        info = plan.solve_fp(dev(u0), None, U)
        assert O.rel_error(host(U), ref) < 1e-10, info
        assert slice_relmax(host(U), ref) < 1e-10, info
        plan.solve_sequential(dev(u0), None, U)
        assert O.rel_error(host(U), ref) < 1e-12


@pytest.mark.parametrize("p", ETD_CASES, ids=ETD_IDS)
def test_etd1_residual_matches_oracle(expd, p):
    sp = O.spec_of(p)
    rng = np.random.default_rng(33)
    u0 = 0.5 * rng.uniform(-1, 1, p.n)
    U = 0.5 * rng.uniform(-1, 1, (p.Nt,) + p.n)
    ref = O.residual(sp, U, O.rhs_known(sp, u0[None], None))
    R = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        plan.residual(dev(u0), None, dev(U), R)
    assert relmax(host(R), ref) < 1e-11


def test_etd1_argument_checks(expd):
    p = ETD_CASES[0]
    with pytest.raises(expd.ExpdError) as ei:
        expd.plan_create(expd.spec_from_problem(p.with_(order=2, Nt=17)))
    assert ei.value.status == expd.ERR_INVALID_ARG
    with pytest.raises(expd.ExpdError) as ei:
        expd.plan_create(expd.spec_from_problem(p, jacobian=expd.JAC_MEAN_U0))
    assert ei.value.status == expd.ERR_INVALID_ARG
    u0 = np.zeros(p.n)
    f = np.zeros((p.Nt,) + p.n)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p)) as plan:
        with pytest.raises(expd.ExpdError) as ei:
            plan.solve_fp(dev(u0), dev(f), U)
        assert ei.value.status == expd.ERR_INVALID_ARG
