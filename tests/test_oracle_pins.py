"""The CPU oracle pinned against things other than itself (runs without a GPU).

Each test names what fixes the expected value: a coefficient the paper prints,
a closed-form solution, a theorem's spectrum, or an independent dense brute
force (explicit L_h, scipy.linalg.expm, explicit alpha-circulant matrices, LU).
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import oracle_checks as C

SPATIAL_CASES = [
    C.spec("periodic", (8,)),
    C.spec("periodic", (4, 6), length=(1.0, 1.5), a=0.02),
    C.spec("dirichlet", (7,)),
    C.spec("dirichlet", (4, 5), a=0.01),
]


def test_bdf_coefficients_match_paper():
    # Eq. (2.2), Eq. (4.1), Eqs. (5.1), (5.3), (5.5), (5.7)
    assert C.check_bdf_golden() == 0.0
    # beta_1 = 1 is the coefficient of dt N(u_n) in Eq. (6.1)
    assert O.bdf_coefficients(1)[1] == 1


@pytest.mark.parametrize("sp", SPATIAL_CASES, ids=lambda s: f"{s.bc}{s.n}")
def test_A_matches_dense_expm(sp):
    # A = exp(dt L_h) (Eq. (2.2)): eigen-symbol path vs expm of the explicit matrix
    assert C.check_A_vs_dense(sp) < 1e-12


def test_periodic_symbol_includes_nyquist():
    sp = C.spec("periodic", (8,), length=(2 * math.pi,), a=1.0, c=0.0)
    ev = np.sort(np.linalg.eigvalsh(O.dense_Lh(sp)))
    assert np.allclose(ev, np.sort(O.spatial_eigenvalues(sp)), atol=1e-12)
    assert np.isclose(ev.min(), -16.0)


@pytest.mark.parametrize("order", [1, 2, 3, 6])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_apply_R_and_rhs_match_dense(order, bc):
    sp = C.spec(bc, (6,), Nt=order + 5, order=order)
    assert C.check_apply_R_vs_dense(sp) < 1e-12
    assert C.check_rhs_vs_dense(sp) < 1e-12


def test_alpha_circulant_structure():
    # Sec. 2 (P_alpha = Gamma^{-1} F^*), Sec. 4 (C_1^alpha entries, lambda_1 = lambda_0^2)
    assert C.check_alpha_circulant() < 1e-13


@pytest.mark.parametrize("order", [1, 2, 6])
@pytest.mark.parametrize("sp0", SPATIAL_CASES, ids=lambda s: f"{s.bc}{s.n}")
def test_precond_three_steps_match_dense_solve(order, sp0):
    # Eq. (3.3) / Eq. (4.5): the three steps equal an LU solve with R_s^alpha
    sp = O.Spec(sp0.bc, sp0.n, sp0.length, sp0.a, sp0.c, "none", sp0.dt, order + 6, 0.07, order)
    assert C.check_precond_vs_dense(sp) < 1e-10


@pytest.mark.parametrize("order", [1, 2, 3, 6])
@pytest.mark.parametrize("bc,nonlin", [("periodic", "none"), ("dirichlet", "none"),
                                       ("periodic", "allen_cahn"), ("dirichlet", "allen_cahn")])
def test_sequential_equals_dense_all_at_once(order, bc, nonlin):
    sp = C.spec(bc, (6,), nonlin=nonlin, Nt=order + 5, order=order, dt=0.02)
    assert C.check_sequential_vs_dense(sp, forcing=True) < 1e-12


def test_sequential_equals_dense_2d_nonlinear():
    sp = C.spec("periodic", (4, 4), length=(1.0, 1.0), a=0.01, c=0.0, nonlin="allen_cahn",
                Nt=8, order=2, dt=0.01)
    assert C.check_sequential_vs_dense(sp, forcing=False) < 1e-12


def test_heat_exact_in_time():
    # spectral exponential Euler reproduces e^{-k^2 t} exactly
    assert C.check_heat_exact() < 1e-13


def test_richardson_iterates_closed_form():
    # u^k_n = (1 - (-q)^k) E^n u0, q = alpha E^Nt / (1 - alpha E^Nt)
    assert C.check_richardson_closed_form() < 1e-13


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_iteration_spectrum_theorems(order, bc):
    # Theorem 3.1 (Eq. (3.6)) and Theorem 4.1
    sp = C.spec(bc, (5,) if bc == "dirichlet" else (6,), Nt=7, order=order, alpha=0.1, a=0.05)
    assert C.check_iteration_spectrum(sp, "theorem") < 1e-8


@pytest.mark.parametrize("order", [3, 6])
def test_iteration_spectrum_order_s(order):
    # generalisation of Theorems 3.1/4.1: roots of zeta^s - sum a_j E^j zeta^{s-j}
    sp = C.spec("dirichlet", (3,), Nt=order + 6, order=order, alpha=0.2, a=0.02, dt=0.1)
    assert C.check_iteration_spectrum(sp, "general") < 1e-6


def test_iteration_spectrum_general_reduces_to_theorems():
    for order in (1, 2):
        sp = C.spec("periodic", (6,), Nt=7, order=order, alpha=0.1)
        got = np.sort_complex(C.predicted_iteration_spectrum(sp))
        want = np.sort_complex(C.theorem_spectrum(sp).astype(complex))
        assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("order", [1, 2, 3])
def test_forced_convergence_order(order):
    # IF-BDF-s with beta_s dt f(t_n) is consistent of order s
    p = C.check_forced_order(order)
    assert abs(p - order) < 0.25, p


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_nonlinear_convergence_order(order):
    # IF-BDF-s with beta_s dt N(u_n) on u' = u - u^3 (exact logistic-type solution)
    p = C.check_nonlinear_order(order)
    assert abs(p - order) < 0.3, p


@pytest.mark.parametrize("order", [1, 2, 6])
def test_dirichlet_single_sine_mode(order):
    assert C.check_dirichlet_single_mode(order) < 1e-13


def test_allen_cahn_constant_state_high_precision():
    # constant state: each grid point follows u_n - dt(u_n - u_n^3) = u_{n-1};
    # compare with a 40-digit scalar Newton solve.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    sp = C.spec("periodic", (4, 4), length=(1.0, 1.0), a=0.01, c=0.0, nonlin="allen_cahn",
                Nt=12, order=1, dt=0.01)
    U = O.sequential_solve(sp, np.full(sp.n, 0.3))
    u = mp.mpf("0.3")
    dt = mp.mpf("0.01")
    for n in range(1, 13):
        w = u
        x = w
        for _ in range(60):
            x = x - (x - dt * (x - x**3) - w) / (1 - dt + 3 * dt * x**2)
        u = x
        assert abs(U[n, 1, 2] - float(u)) < 1e-16


def test_thm21_contraction_bound():
    r = C.check_thm21_contraction()
    assert r <= 1.0 + 1e-9, r


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_gmres_terminates_thm33(bc):
    # Theorem 3.3: at most Nx + 1 iterations (first order)
    sp = C.spec(bc, (5,) if bc == "dirichlet" else (6,), Nt=9, order=1, alpha=0.5, a=0.3)
    its, res = C.check_gmres_terminates(sp)
    assert its <= int(np.prod(sp.n)) + 1
    assert res.history[-1] < 1e-12


def test_gmres_terminates_thm43():
    # Theorem 4.3: at most 2 Nx + 1 iterations (second order)
    sp = C.spec("dirichlet", (4,), Nt=9, order=2, alpha=0.5, a=0.3)
    its, res = C.check_gmres_terminates(sp)
    assert its <= 2 * int(np.prod(sp.n)) + 1


def test_gmres_elman_bound_thm314():
    sp = C.spec("dirichlet", (8,), Nt=10, order=1, alpha=0.2, a=0.01, c=0.0)
    assert C.check_gmres_elman(sp) <= 1.0 + 1e-12


@pytest.mark.parametrize("order", [1, 2, 6])
def test_gmres_and_richardson_reach_sequential(order):
    sp = C.spec("periodic", (4, 4), length=(1.0, 1.0), a=0.05, c=0.1, Nt=order + 9,
                order=order, alpha=1e-3, dt=0.02)
    rng = np.random.default_rng(order)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    ref = O.sequential_solve(sp, u0, f)
    g = O.gmres(sp, u0, f, tol=1e-13)
    r = O.richardson(sp, u0, f, max_iter=8)
    assert O.rel_error(g.U[1:], ref[1:]) < 1e-12
    assert O.rel_error(r.U[1:], ref[1:]) < 1e-12


def test_lagged_nonlinear_richardson_reaches_sequential():
    # Eqs. (7.3)-(7.4) and their order-s extension
    for order in (1, 2, 6):
        sp = C.spec("periodic", (8, 8), length=(1.0, 1.0), a=0.0025, c=0.0,
                    nonlin="allen_cahn", Nt=order + 15, order=order, alpha=1e-3, dt=1e-3)
        u0 = np.random.default_rng(10 + order).uniform(-0.9, 0.9, sp.n)
        ref = O.sequential_solve(sp, u0)
        r = O.richardson(sp, u0, max_iter=30, tol=1e-15)
        assert O.rel_error(r.U[1:], ref[1:]) < 1e-12


def test_one_iteration_claim_long_window():
    # Sec. 7.1: T = 64 with dt = h = 1/128, 1,048,576 unknowns, one iteration.
    claims = {}
    with open(C.os.path.join(C.GOLDEN, "paper_claims.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                claims[k] = float(v)
    dt = claims["one_iteration_dt"]
    Nt = int(round(claims["one_iteration_T"] / dt))
    nx = int(claims["one_iteration_unknowns"]) // Nt
    L = (nx + 1) * dt                          # h = L/(nx+1) = 1/128
    sp = O.Spec("dirichlet", (nx,), (L,), claims["one_iteration_a"], claims["one_iteration_c"],
                "none", dt, Nt, claims["alpha_opt"], 1)
    x = np.arange(1, nx + 1) * L / (nx + 1)
    u0 = np.exp(-30 * (x - L / 2) ** 2)
    assert nx * Nt == 1048576
    ref = O.sequential_solve(sp, u0)
    r = O.richardson(sp, u0, max_iter=1)
    assert O.rel_error(r.U[1:], ref[1:]) < claims["one_iteration_tol"]


@pytest.mark.parametrize("eigs", [(3.0,) * 5, (2.0, 2.0, 5.0, 5.0, 5.0), (2.0, 2.0, 5.0, 5.0, 5.0, -1.5),
                                  (1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0)])
def test_bicgstab_terminates_with_the_minimal_polynomial(eigs):
    # BiCG-type finite termination: d distinct eigenvalues -> exact after d steps
    hist, d, err = C.check_bicgstab_minimal_polynomial(eigs)
    assert len(hist) == d + 1
    assert hist[d] < 1e-10 and err < 1e-10, (hist, err)


@pytest.mark.parametrize("order", [1, 2, 6])
def test_bicgstab_reaches_sequential(order):
    sp = C.spec("periodic", (4, 4), length=(1.0, 1.0), a=0.05, c=0.1, Nt=order + 9,
                order=order, alpha=1e-3, dt=0.02)
    err, res = C.check_bicgstab_reaches_sequential(sp)
    assert err < 1e-12
    assert res.iterations <= 6          # preconditioned spectrum clustered at 1 (Lemma 3.4)


@pytest.mark.parametrize("bc,order", [("periodic", 1), ("dirichlet", 2), ("periodic", 6)])
def test_shifted_preconditioner_matches_dense(bc, order):
    # Step (b) of the inexact Newton variant (Eq. (6.5)) with a scalar Jacobian
    sp = C.spec(bc, (5,) if bc == "dirichlet" else (6,), Nt=order + 7, order=order, alpha=0.05, a=0.3)
    assert C.check_precond_shift_vs_dense(sp) < 1e-11


@pytest.mark.parametrize("order", [1, 2, 6])
def test_mean_jacobian_reaches_sequential(order):
    sp = C.spec("periodic", (8, 8), length=(1.0, 1.0), a=0.0025, c=0.0, nonlin="allen_cahn",
                Nt=order + 15, order=order, alpha=1e-3, dt=1e-3)
    u0 = np.random.default_rng(20 + order).uniform(-0.9, 0.9, sp.n)
    ref = O.sequential_solve(sp, u0)
    r = O.richardson(sp, u0, max_iter=40, tol=1e-14, jacobian="mean_u0")
    assert O.rel_error(r.U[1:], ref[1:]) < 1e-12


def test_mean_jacobian_contracts_faster_near_uniform_state():
    # near a uniform state the mean of N'(u_0) is the Jacobian: the inexact
    # Newton iteration contracts much faster than the lagged one
    rho_lag, rho_newton = C.check_mean_jacobian_contraction()
    assert rho_newton < 0.2 * rho_lag, (rho_lag, rho_newton)


# ------------------------------------------ advection-diffusion (periodic) --
ADV_SPECS = [C.adv_spec(), C.adv_spec(n=(4, 6), length=(1.0, 1.5), b=(0.7, -0.4), order=2, Nt=10),
             C.adv_spec(n=(6,), b=(-1.3,), order=6, Nt=14)]


@pytest.mark.parametrize("sp", ADV_SPECS, ids=["1d_s1", "2d_s2", "1d_s6"])
def test_advection_symbol_and_system_vs_dense(sp):
    # the complex symbol -a|k|^2 - i b.k - c against expm of the explicit
    # a D2 - b.D1 - c (spectral sinc derivative matrices), and the all-at-once
    # operators built on it
    assert C.check_A_vs_dense(sp) < 1e-12
    assert C.check_apply_R_vs_dense(sp) < 1e-12
    assert C.check_precond_vs_dense(sp) < 1e-10
    assert C.check_sequential_vs_dense(sp) < 1e-12
    assert C.check_rhs_vs_dense(sp) < 1e-12


def test_advection_exact_transport():
    # spectral exponential Euler transports and damps each Fourier mode exactly
    assert C.check_advection_exact() < 1e-12


@pytest.mark.parametrize("order", [1, 2, 6])
def test_advection_solvers_reach_sequential(order):
    sp = C.adv_spec(n=(8, 8), length=(1.0, 1.0), b=(2.0, -1.0), order=order, Nt=order + 11, a=0.01, alpha=1e-3, dt=0.01)
    rng = np.random.default_rng(30 + order)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    ref = O.sequential_solve(sp, u0, f)[1:]
    assert O.rel_error(O.richardson(sp, u0, f, max_iter=12).U[1:], ref) < 1e-11
    assert O.rel_error(O.gmres(sp, u0, f, tol=1e-13).U[1:], ref) < 1e-11
    assert O.rel_error(O.bicgstab(sp, u0, f, tol=1e-13).U[1:], ref) < 1e-11


def test_linear_guess_solves_the_homogeneous_scheme():
    # the default initial iterate of the fixed point: exact for N = 0, f = 0
    assert C.check_linear_guess_is_homogeneous_solution() < 1e-12


def test_linear_guess_reaches_the_same_fixed_point_one_sweep_sooner():
    # Allen-Cahn: both initial iterates converge to the same fixed point; the
    # zero iterate's first sweep produces (up to the alpha perturbation) what
    # the linear guess already is, so the histories are shifted by one sweep
    sp = C.spec("periodic", (16, 16), length=(1.0, 1.0), a=0.0025, c=0.0, nonlin="allen_cahn",
                Nt=32, order=1, alpha=1e-3, dt=1e-3)
    u0 = np.random.default_rng(21).uniform(-0.9, 0.9, sp.n)
    rz = O.richardson(sp, u0, max_iter=8, init="zero")
    rl = O.richardson(sp, u0, max_iter=8, init="linear")
    assert O.rel_error(rl.U[1:], rz.U[1:]) < 1e-12
    for k in range(1, 5):
        assert rl.history[k - 1] < 3.0 * rz.history[k]


# ------------------------------------------------------------------- ETD1 --
# u_n = A u_{n-1} + dt phi_1(dt L_h) N(u_{n-1}), the first-order ETD form of
# the nonlinear term that Sec. 6 names beside its integrating-factor form.
def test_phi1_scalar_against_high_precision():
    assert C.check_phi1_scalar() < 4e-16


@pytest.mark.parametrize("sp", [C.etd_spec("periodic", (8,)), C.etd_spec("dirichlet", (7,)),
                                C.etd_spec("periodic", (4, 6)), C.etd_spec("dirichlet", (5, 4))],
                         ids=["p1d", "d1d", "p2d", "d2d"])
def test_phi1_matches_dense_augmented_expm(sp):
    assert C.check_phi1_vs_dense(sp) < 1e-12


@pytest.mark.parametrize("sp", [C.etd_spec("periodic", (8,)), C.etd_spec("dirichlet", (5, 4), Nt=5)],
                         ids=["p1d", "d2d"])
def test_etd1_sequential_equals_dense_all_at_once(sp):
    assert C.check_etd1_sequential_vs_dense(sp) < 1e-12


def test_etd1_first_order_convergence():
    p = C.check_etd1_order()
    assert abs(p - 1.0) < 0.1, p


@pytest.mark.parametrize("sp", [C.etd_spec("periodic", (8,), Nt=10), C.etd_spec("dirichlet", (6, 5), Nt=8)],
                         ids=["p1d", "d2d"])
def test_etd1_richardson_reaches_sequential(sp):
    assert C.check_etd1_richardson_reaches_sequential(sp) < 1e-12


# --------------------------------------------------- complex states (Sec. 7) --
SE_SPECS = [
    C.se_spec("dirichlet", (7,), 1j, 2j, Nt=8, order=1),
    C.se_spec("dirichlet", (3, 4), 1j, 200j, Nt=9, order=2, dt=0.05),
    C.se_spec("dirichlet", (5,), 0.3 + 1j, 0.1 + 2j, Nt=14, order=6, dt=0.02),
    C.se_spec("periodic", (8,), 1j, 2j, Nt=8, order=1),
    C.se_spec("periodic", (4, 6), 0.05 + 1j, 1j, Nt=9, order=2, length=(1.0, 1.5)),
]
SE_IDS = ["d1_s1", "d2_s2_c200i", "d1_s6_mixed", "p1_s1", "p2_s2"]


@pytest.mark.parametrize("sp", SE_SPECS, ids=SE_IDS)
def test_complex_A_matches_dense_expm(sp):
    assert C.check_complex_A_vs_dense(sp) < 1e-12


@pytest.mark.parametrize("sp", SE_SPECS, ids=SE_IDS)
def test_complex_precond_matches_dense(sp):
    assert C.check_complex_precond_vs_dense(sp) < 1e-11


@pytest.mark.parametrize("sp", SE_SPECS, ids=SE_IDS)
def test_complex_sequential_matches_dense(sp):
    assert C.check_complex_sequential_vs_dense(sp) < 1e-11


def test_schrodinger_sine_mode_closed_form():
    assert C.check_schrodinger_sine_mode() < 1e-13


@pytest.mark.parametrize("sp", [C.se_spec("dirichlet", (9,), 1j, 2j, Nt=12, order=1),
                                C.se_spec("dirichlet", (3, 3), 1j, 200j, Nt=12, order=2),
                                C.se_spec("periodic", (8,), 1j, 0.5j, Nt=12, order=6, dt=0.01)],
                         ids=["d_s1", "d2_s2", "p_s6"])
def test_unitary_propagator_keeps_norm(sp):
    assert C.check_unitary_norm(sp) < 1e-12


@pytest.mark.parametrize("sp", SE_SPECS[:3], ids=SE_IDS[:3])
def test_complex_gmres_matches_dense(sp):
    err, res = C.check_complex_gmres_vs_dense(sp)
    assert err < 1e-11
    assert res.history[-1] < 1e-13


@pytest.mark.parametrize("sp", SE_SPECS[:3], ids=SE_IDS[:3])
def test_complex_bicgstab_matches_dense(sp):
    err, _ = C.check_complex_bicgstab_vs_dense(sp)
    assert err < 1e-11


@pytest.mark.parametrize("Nt", (50, 100, 200))
def test_schrodinger_1d_gmres_one_iteration(Nt):
    # Sec. 7: GMRES with the Exp-ParaDiag preconditioner converges in one
    # iteration on the 1D Schrodinger equation (h = 1/128, dt = 0.01,
    # alpha_opt, u_0 = sin(pi x)) for every window length: u_0 is an
    # eigenvector of L_h, so the first residual is an eigenvector of the
    # preconditioned operator (complex GMRES; a real GMRES on the real and
    # imaginary parts would need two steps)
    from paper_2603_04350_gb300 import inputs as I
    errs = C.schrodinger_gmres_errors(I.SCHRODINGER_1D.with_(Nt=Nt), 1)
    assert errs[0] < 1e-10


@pytest.mark.parametrize("Nt", (20, 80))
def test_schrodinger_2d_gmres_three_iterations(Nt):
    # Sec. 7: BDF2 GMRES on the 2D Schrodinger equation (h = 1/40, dt = 0.05,
    # c = 200i, the Gaussian wave packet) reaches the 1e-10 error in three
    # iterations whatever the window length
    from paper_2603_04350_gb300 import inputs as I
    errs = C.schrodinger_gmres_errors(I.SCHRODINGER_2D.with_(Nt=Nt), 3)
    assert errs[1] > 1e-10 and errs[2] < 1e-10


# ------------------------------------------------------- Neumann grids (Sec. 7) --
NEU_SPECS = [
    C.neu_spec((8,), order=1),
    C.neu_spec((5, 6), order=2),
    C.neu_spec((7,), order=6, Nt=14, dt=0.02),
    C.neu_spec((6, 5), a=0.01, c=0.0, nonlin="allen_cahn", order=2, dt=0.02),
]
NEU_IDS = ["n1_s1", "n2_s2", "n1_s6", "n2_ac_s2"]


@pytest.mark.parametrize("sp", NEU_SPECS, ids=NEU_IDS)
def test_neumann_A_matches_dense_expm(sp):
    assert C.check_A_vs_dense(sp) < 1e-12


@pytest.mark.parametrize("sp", NEU_SPECS, ids=NEU_IDS)
def test_neumann_precond_and_R_match_dense(sp):
    assert C.check_precond_vs_dense(sp) < 1e-11
    assert C.check_apply_R_vs_dense(sp) < 1e-12


@pytest.mark.parametrize("sp", NEU_SPECS, ids=NEU_IDS)
def test_neumann_sequential_matches_dense(sp):
    assert C.check_sequential_vs_dense(sp) < 1e-11


def test_neumann_mass_conservation():
    assert C.check_neumann_mass() < 1e-13


def test_neumann_cosine_mode_closed_form():
    assert C.check_neumann_cosine_mode() < 1e-13


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 4.0)])
def test_neumann_allen_cahn_exact_solution_order(order, ratio):
    # Sec. 7's Neumann Allen-Cahn problem with a manufactured exact solution:
    # halving dt divides the error by 2 (s = 1) and about 4 (s = 2)
    errs = C.neumann_allen_cahn_errors(order, steps=(25, 50, 100))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[0] < 3e-4
    assert all(abs(r - ratio) < 0.15 * ratio for r in rates)


def test_neumann_gmres_and_richardson_reach_dense():
    sp = C.neu_spec((5, 4), order=2, Nt=10, alpha=0.05)
    rng = np.random.default_rng(31)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    ref = O.dense_solve(sp, u0, f)[1:]
    assert O.rel_error(O.gmres(sp, u0, f, tol=1e-13).U[1:], ref) < 1e-11
    assert O.rel_error(O.richardson(sp, u0, f, max_iter=60, tol=1e-14).U[1:], ref) < 1e-11

@pytest.mark.parametrize("bc,n,order,Nt", [("dirichlet", (9,), 1, 6), ("dirichlet", (7, 5), 2, 12),
                                           ("dirichlet", (9,), 6, 13), ("neumann", (8,), 3, 10),
                                           ("periodic", (8,), 2, 9)])
def test_wraparound_identity_of_the_krylov_operator(bc, n, order, Nt):
    # the form the tensor-core time kernel applies the Krylov operator in
    assert C.check_wraparound_identity(bc, n, order, Nt) < 1e-12


@pytest.mark.parametrize("n", [8, 12, 64])
def test_dst_mirror_symmetry_and_fold(n):
    # the symmetry the folded tensor-core sine transform relies on
    assert C.check_dst_mirror_fold(n) < 1e-13
