"""Plant plausible mistakes in the CPU oracle and check that a pin catches each.

A mistake is planted by monkeypatching one oracle function for the duration of
one test (on the CPU only); the matching pin from tests/oracle_checks.py must
then exceed the tolerance that tests/test_oracle_pins.py asserts.
"""
import numpy as np
import pytest

import oracle as O
import oracle.expd_oracle as E
from tests import oracle_checks as C


def patch(monkeypatch, name, fn):
    monkeypatch.setattr(E, name, fn)
    monkeypatch.setattr(O, name, fn)


def precond_variant(conj_omega=False, gamma_den=0, no_power=False, drop_gamma_inverse=False):
    def precond_apply(sp, r):
        Ns = sp.Ns
        a, _ = E.bdf_float(sp.order)
        gam = (sp.alpha ** (np.arange(Ns) / (Ns + gamma_den))).reshape((Ns,) + (1,) * sp.ndim)
        lam = E.time_eigenvalues(sp)
        mu = E.spatial_eigenvalues(sp)
        fwd = np.fft.fft if conj_omega else np.fft.ifft
        inv = np.fft.ifft if conj_omega else np.fft.fft
        scale = (1.0 / Ns) if conj_omega else 1.0
        Sa = np.sqrt(Ns) * fwd(gam * r, axis=0) * scale
        Sb = np.empty_like(Sa)
        for n in range(Ns):
            d = np.ones(sp.n, dtype=complex)
            for j in range(1, sp.order + 1):
                d -= a[j - 1] * (lam[n] if no_power else lam[n] ** j) * np.exp(j * sp.dt * mu)
            Sb[n] = E.from_eigen(sp, E.to_eigen(sp, Sa[n]) / d)
        s = inv(Sb, axis=0) / np.sqrt(Ns) / scale
        if not drop_gamma_inverse:
            s = s / gam
        return s.real
    return precond_apply


SP6 = O.Spec("periodic", (4, 6), (1.0, 1.5), 0.02, 0.1, "none", 0.05, 12, 0.07, 6)
SP2 = O.Spec("dirichlet", (5,), (1.0,), 0.3, 0.1, "none", 0.05, 9, 0.07, 2)


@pytest.mark.parametrize("kw", [dict(conj_omega=True), dict(gamma_den=-1), dict(no_power=True),
                                dict(drop_gamma_inverse=True)],
                         ids=["omega_sign", "gamma_root", "lambda_power", "gamma_inverse"])
def test_planted_precond_mistakes_are_caught(monkeypatch, kw):
    patch(monkeypatch, "precond_apply", precond_variant(**kw))
    assert max(C.check_precond_vs_dense(SP6), C.check_precond_vs_dense(SP2)) > 1e-6


def test_planted_wrong_shift_direction_is_caught(monkeypatch):
    def apply_R(sp, V):
        a, _ = E.bdf_float(sp.order)
        out = V.copy()
        for i in range(sp.Ns):
            for j in range(1, sp.order + 1):
                if i + j < sp.Ns:                      # transposed shift
                    out[i] -= a[j - 1] * E.apply_A_power(sp, V[i + j], j)
        return out
    patch(monkeypatch, "apply_R", apply_R)
    assert C.check_apply_R_vs_dense(SP2) > 1e-3


def test_planted_dropped_startup_term_is_caught(monkeypatch):
    orig = E.rhs_known

    def rhs_known(sp, U_start, f):
        return orig(sp, U_start[:1].repeat(sp.order, axis=0) * 0 + U_start[-1:], f)
    patch(monkeypatch, "rhs_known", rhs_known)
    sp = C.spec("periodic", (6,), Nt=9, order=3)
    assert C.check_rhs_vs_dense(sp) > 1e-3


def test_planted_wrong_nyquist_symbol_is_caught(monkeypatch):
    def spatial_eigenvalues(sp):
        parts = []
        for n, L in zip(sp.n, sp.length):
            k = np.arange(n)                            # forgot the negative frequencies
            parts.append(-(2.0 * np.pi * k / L) ** 2)
        return sp.a * sum(np.meshgrid(*parts, indexing="ij")) - sp.c
    patch(monkeypatch, "spatial_eigenvalues", spatial_eigenvalues)
    assert C.check_A_vs_dense(C.spec("periodic", (8,))) > 1e-3


def test_planted_missing_beta_on_source_is_caught(monkeypatch):
    def step_rhs(sp, U, n, q, f):
        a, beta = E.bdf_float(q)
        w = np.zeros(sp.n)
        for j in range(1, q + 1):
            w += a[j - 1] * E.apply_A_power(sp, U[n - j], j)
        if f is not None:
            w += sp.dt * f[n - 1]                      # beta dropped
        return w
    patch(monkeypatch, "step_rhs", step_rhs)
    assert abs(C.check_forced_order(2) - 2) > 0.5


def test_planted_wrong_bdf_coefficient_is_caught(monkeypatch):
    orig = E.bdf_coefficients

    def bdf_coefficients(s):
        a, beta = orig(s)
        if s >= 2:
            a = list(a)
            a[1] = -a[1]
        return a, beta
    patch(monkeypatch, "bdf_coefficients", bdf_coefficients)
    assert C.check_bdf_golden() > 0


def test_planted_wrong_nonlinear_sign_is_caught(monkeypatch):
    def nonlinearity(sp, u):
        return u + u**3 if sp.nonlin == "allen_cahn" else np.zeros_like(u)
    patch(monkeypatch, "nonlinearity", nonlinearity)
    sp = C.spec("periodic", (6,), nonlin="allen_cahn", Nt=8, order=1, dt=0.02)
    # sequential (pointwise Newton) vs dense Newton: both use their own N, so
    # the Richardson fixed point (which uses nonlinearity) moves off the
    # sequential solution.
    u0 = np.random.default_rng(0).uniform(-0.8, 0.8, sp.n)
    ref = O.sequential_solve(sp, u0)
    r = O.richardson(sp, u0, max_iter=30)
    assert O.rel_error(r.U[1:], ref[1:]) > 1e-6


@pytest.mark.parametrize("mistake", ["beta_sign", "omega_dropped"])
def test_planted_bicgstab_mistakes_are_caught(monkeypatch, mistake):
    def bicgstab_solve(matvec, b, tol, max_iter):
        x = np.zeros_like(b)
        r = b.copy()
        rhat = r.copy()
        rho = alpha = omega = 1.0
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        hist = [1.0]
        for _ in range(max_iter):
            rho_new = float(np.dot(rhat, r))
            beta = (rho_new / rho) * (alpha / omega)
            if mistake == "beta_sign":
                beta = -beta
            p = r + beta * (p - omega * v)
            v = matvec(p)
            alpha = rho_new / float(np.dot(rhat, v))
            s = r - alpha * v
            t = matvec(s)
            omega = float(np.dot(t, s)) / float(np.dot(t, t))
            x = x + alpha * p + (0.0 if mistake == "omega_dropped" else omega) * s
            r = s - omega * t
            rho = rho_new
            hist.append(float(np.linalg.norm(r)) / np.linalg.norm(b))
        return x, hist
    patch(monkeypatch, "bicgstab_solve", bicgstab_solve)
    hist, d, err = C.check_bicgstab_minimal_polynomial((2.0, 2.0, 5.0, 5.0, 5.0, -1.5))
    assert hist[d] > 1e-6 or err > 1e-6


def test_planted_jacobian_shift_sign_is_caught(monkeypatch):
    real = E.jacobian_shift
    patch(monkeypatch, "jacobian_shift", lambda sp, u0: -real(sp, u0))
    rho_lag, rho_newton = C.check_mean_jacobian_contraction()
    assert not rho_newton < 0.2 * rho_lag


def test_planted_advection_sign_is_caught(monkeypatch):
    real = E.spatial_eigenvalues
    patch(monkeypatch, "spatial_eigenvalues", lambda sp: np.conj(real(sp)))
    assert C.check_advection_exact() > 1e-3


def test_planted_linear_guess_power_is_caught(monkeypatch):
    # off by one in the propagation power: A^k instead of A^(k+1)
    def linear_guess(sp, U_start):
        u_last = U_start[sp.order - 1]
        return np.stack([E.apply_A_power(sp, u_last, k) for k in range(sp.Ns)])
    patch(monkeypatch, "linear_guess", linear_guess)
    assert C.check_linear_guess_is_homogeneous_solution() > 1e-6


# ------------------------------------------------------------------- ETD1 --
ETD_P = C.etd_spec("periodic", (8,), Nt=10)
ETD_D = C.etd_spec("dirichlet", (5, 4), Nt=5)


@pytest.mark.parametrize("kind", ["phi_is_one", "no_dt"])
def test_planted_phi1_mistakes_are_caught(monkeypatch, kind):
    def apply_phi1(sp, u):
        mu = E.spatial_eigenvalues(sp)
        sym = np.ones_like(mu) if kind == "phi_is_one" else E.phi1(sp.dt * mu)
        scale = sp.dt if kind == "phi_is_one" else 1.0
        return E.from_eigen(sp, scale * sym * E.to_eigen(sp, u)).real
    patch(monkeypatch, "apply_phi1", apply_phi1)
    assert max(C.check_phi1_vs_dense(ETD_P), C.check_phi1_vs_dense(ETD_D)) > 1e-3


def test_planted_etd1_nonlinearity_at_the_propagated_state_is_caught(monkeypatch):
    def etd1_step(sp, u_prev):
        w = E.apply_A_power(sp, u_prev, 1)
        return w + E.apply_phi1(sp, E.nonlinearity(sp, w))     # N(A u) instead of N(u)
    patch(monkeypatch, "etd1_step", etd1_step)
    assert C.check_etd1_sequential_vs_dense(ETD_P) > 1e-6


def test_planted_etd1_residual_on_the_same_slice_is_caught(monkeypatch):
    orig = E.residual

    def residual(sp, V, b):
        r = b - E.apply_R(sp, V)
        for i in range(1, sp.Ns):
            r[i] += E.apply_phi1(sp, E.nonlinearity(sp, V[i]))  # slice i instead of i - 1
        return r if E.is_etd1(sp) else orig(sp, V, b)
    patch(monkeypatch, "residual", residual)
    assert C.check_etd1_richardson_reaches_sequential(ETD_P) > 1e-6


# ------------------------------------------------------------ complex states --
def _patched_source(monkeypatch, name, old, new):
    """Plant a mistake by editing one line of an oracle function's source."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(E, name)))
    assert old in src
    ns = dict(vars(E))
    exec(compile(src.replace(old, new), E.__file__, "exec"), ns)
    patch(monkeypatch, name, ns[name])


SE_D1 = C.se_spec("dirichlet", (7,), 1j, 2j, Nt=8, order=1)
SE_D2 = C.se_spec("dirichlet", (3, 4), 1j, 200j, Nt=9, order=2)


def test_planted_unconjugated_gmres_product_is_caught(monkeypatch):
    # the bilinear sum v w in place of the Hermitian sum conj(v) w
    _patched_source(monkeypatch, "gmres", "H[i, j] = np.vdot(Vb[i], w)", "H[i, j] = np.dot(Vb[i], w)")
    err, _ = C.check_complex_gmres_vs_dense(SE_D2)
    assert err > 1e-6


def test_planted_real_gmres_coefficients_are_caught(monkeypatch):
    # GMRES on the real and imaginary parts as a real vector (real projection
    # coefficients): correct in the limit, but no longer one iteration on the
    # 1D Schrodinger problem of Sec. 7
    _patched_source(monkeypatch, "gmres", "H[i, j] = np.vdot(Vb[i], w)", "H[i, j] = np.vdot(Vb[i], w).real")
    from paper_2603_04350_gb300 import inputs as I
    assert C.schrodinger_gmres_errors(I.SCHRODINGER_1D.with_(Nt=50), 1)[0] > 1e-6


def test_planted_real_part_of_complex_preconditioner_is_caught(monkeypatch):
    _patched_source(monkeypatch, "precond_apply", "return s if sp.complex_state else s.real", "return s.real")
    assert C.check_complex_precond_vs_dense(SE_D1) > 1e-3


def test_planted_conjugated_symbol_is_caught(monkeypatch):
    orig = E.spatial_eigenvalues

    def spatial_eigenvalues(sp):
        return np.conj(orig(sp))
    patch(monkeypatch, "spatial_eigenvalues", spatial_eigenvalues)
    assert C.check_schrodinger_sine_mode() > 1e-3


def test_planted_neumann_dirichlet_index_is_caught(monkeypatch):
    # the Neumann symbol evaluated at k + 1 (the Dirichlet sine index)
    _patched_source(monkeypatch, "spatial_eigenvalues", "k = np.arange(n)\n", "k = np.arange(1, n + 1)\n")
    assert C.check_A_vs_dense(C.neu_spec((8,))) > 1e-3


def test_planted_neumann_wrong_cosine_transform_is_caught(monkeypatch):
    # the DCT-I in place of the DCT-II (vertex instead of cell-centred basis)
    _patched_source(monkeypatch, "to_eigen", 'return scipy.fft.dctn(u, type=2, axes=ax, norm="ortho")',
                    'return scipy.fft.dctn(u, type=1, axes=ax, norm="ortho")')
    assert C.check_A_vs_dense(C.neu_spec((8,))) > 1e-3
