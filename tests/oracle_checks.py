"""Pin checks for the CPU oracle, written as functions that return an error
measure so that tests/test_oracle_pins.py can assert on them and
tests/test_oracle_planted.py can show that a planted mistake trips them.

Every check compares the oracle with something other than itself: a closed
form, a value printed in the paper, an independent dense brute force (explicit
L_h, scipy.linalg.expm, explicit alpha-circulant matrices, LU), or a textbook
ODE solution.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def spec(bc="periodic", n=(8,), length=None, a=0.3, c=0.1, nonlin="none", dt=0.05, Nt=8,
         alpha=0.05, order=1):
    if length is None:
        length = tuple(2 * math.pi if bc == "periodic" else 1.0 for _ in n)
    return O.Spec(bc, tuple(n), tuple(length), a, c, nonlin, dt, Nt, alpha, order)


def rng_field(sp, seed, lead=()):
    return np.random.default_rng(seed).standard_normal(tuple(lead) + sp.n)


# --- printed coefficients -------------------------------------------------
def read_golden_bdf():
    rows = {}
    with open(os.path.join(GOLDEN, "bdf_coefficients.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            tok = line.split()
            s = int(tok[0])
            rows[s] = [Fraction(t) for t in tok[1:1 + s]]
    return rows


def check_bdf_golden():
    """Max |a_j(oracle) - a_j(paper)| over s = 1..6 (exact fractions)."""
    worst = Fraction(0)
    for s, printed in read_golden_bdf().items():
        a, _ = O.bdf_coefficients(s)
        worst = max(worst, max(abs(x - y) for x, y in zip(a, printed)))
    return float(worst)


# --- spatial operator -----------------------------------------------------
def check_A_vs_dense(sp, seed=0):
    """Relative difference of the oracle's A^j u (eigen-symbol path) and the
    dense expm of the explicit L_h, j = 1..3."""
    A = O.dense_A(sp)
    u = rng_field(sp, seed)
    worst = 0.0
    Aj = np.eye(A.shape[0])
    for j in range(1, 4):
        Aj = Aj @ A
        ref = (Aj @ u.ravel()).reshape(sp.n)
        got = O.apply_A_power(sp, u, j)
        worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
    return worst


# --- all-at-once pieces ---------------------------------------------------
def check_apply_R_vs_dense(sp, seed=1):
    V = rng_field(sp, seed, (sp.Ns,))
    ref = (O.dense_R(sp) @ V.ravel()).reshape(V.shape)
    return np.abs(O.apply_R(sp, V) - ref).max() / np.abs(ref).max()


def check_precond_vs_dense(sp, seed=2):
    r = rng_field(sp, seed, (sp.Ns,))
    ref = O.dense_precond_apply(sp, r)
    return np.abs(O.precond_apply(sp, r) - ref).max() / np.abs(ref).max()


def check_sequential_vs_dense(sp, seed=3, forcing=True):
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-0.8, 0.8, size=sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n) if forcing else None
    U = O.sequential_solve(sp, u0, f)
    Ud = O.dense_solve(sp, u0, f)
    return O.rel_error(U[1:], Ud[1:])


def check_rhs_vs_dense(sp, seed=4):
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    Us = O.startup_values(sp, u0, f)
    ref = O.dense_rhs(sp, Us, f).reshape((sp.Ns,) + sp.n)
    return np.abs(O.rhs_known(sp, Us, f) - ref).max() / np.abs(ref).max()


# --- alpha-circulant structure -------------------------------------------
def check_alpha_circulant(N=7, alpha=0.3):
    """C_0^alpha = P_alpha D_0 P_alpha^{-1} with P_alpha = Gamma^{-1} F^* (Sec. 2),
    lambda_{1,n} = lambda_{0,n}^2 diagonalises C_1^alpha (Sec. 4), C_1^alpha
    has alpha exactly at (1, N-1), (2, N) (1-based), and C_j^alpha =
    (C_0^alpha)^(j+1)."""
    sp = O.Spec("periodic", (4,), (1.0,), 1.0, 0.0, "none", 0.1, N, alpha, 1)
    gam = O.gamma_alpha(sp)
    lam = O.time_eigenvalues(sp)
    w = np.exp(2j * np.pi / N)
    F = np.array([[w ** (l * k) for k in range(N)] for l in range(N)]) / np.sqrt(N)
    P = np.diag(1.0 / gam) @ F.conj().T
    Pinv = np.linalg.inv(P)
    C0 = O.shift_matrix(N, 0, alpha)
    C1 = O.shift_matrix(N, 1, alpha)
    err = np.abs(P @ np.diag(lam) @ Pinv - C0).max()
    err = max(err, np.abs(P @ np.diag(lam**2) @ Pinv - C1).max())
    printed = np.zeros((N, N))
    for r in range(2, N):
        printed[r, r - 2] = 1.0
    printed[0, N - 2] = alpha
    printed[1, N - 1] = alpha
    err = max(err, np.abs(C1 - printed).max())
    for j in range(6):
        err = max(err, np.abs(O.shift_matrix(N, j, alpha)
                              - np.linalg.matrix_power(C0, j + 1)).max())
    # the printed lambda_{1,n} formula
    lam1 = alpha ** (2.0 / N) * np.exp(4j * np.pi * np.arange(N) / N)
    err = max(err, np.abs(lam1 - lam**2).max())
    return err


# --- spectra of the iteration matrix -------------------------------------
def predicted_iteration_spectrum(sp):
    """Non-zero eigenvalues -alpha z^N/(1 - alpha z^N) per spatial mode, z the
    roots of zeta^s - sum_j a_j E^j zeta^(s-j), N = Ns.  For s = 1 this is
    Theorem 3.1 (Eq. (3.6)); for s = 2 Theorem 4.1 (z = E, E/3)."""
    mu = O.spatial_eigenvalues(sp).ravel()
    a, _ = O.bdf_float(sp.order)
    out = []
    for m in mu:
        E = math.exp(sp.dt * m)
        coef = [1.0] + [-a[j - 1] * E**j for j in range(1, sp.order + 1)]
        for z in np.roots(coef):
            zN = z ** sp.Ns
            out.append(-sp.alpha * zN / (1 - sp.alpha * zN))
    return np.array(out)


def theorem_spectrum(sp):
    """The printed closed forms: Theorem 3.1 (s = 1) and Theorem 4.1 (s = 2)."""
    mu = O.spatial_eigenvalues(sp).ravel()
    out = []
    for m in mu:
        z = sp.dt * m
        if sp.order == 1:
            q = sp.alpha * math.exp(z * sp.Nt)
            out.append(-q / (1 - q))
        elif sp.order == 2:
            N1 = sp.Nt - 1
            q1 = sp.alpha * math.exp(N1 * z)
            q2 = sp.alpha * (math.exp(z) / 3.0) ** N1
            out += [-q1 / (1 - q1), -q2 / (1 - q2)]
        else:
            raise ValueError
    return np.array(out)


def match_multisets(got, want):
    """Max distance after greedy matching of two small complex multisets."""
    got = list(got)
    worst = 0.0
    for w in want:
        i = int(np.argmin([abs(g - w) for g in got]))
        worst = max(worst, abs(got[i] - w))
        got.pop(i)
    return worst


def check_iteration_spectrum(sp, closed_form="theorem"):
    """Distance between the dense iteration matrix's non-zero spectrum and the
    predicted one; plus the size of the eigenvalues that must be zero."""
    ev = np.linalg.eigvals(O.dense_iteration_matrix(sp))
    want = theorem_spectrum(sp) if closed_form == "theorem" else predicted_iteration_spectrum(sp)
    order = np.argsort(-np.abs(ev))
    big = ev[order[: len(want)]]
    rest = ev[order[len(want):]]
    scale = max(1e-300, np.abs(want).max())
    return max(match_multisets(big, want) / scale, (np.abs(rest).max() if rest.size else 0.0) / scale)


# --- closed-form solutions ----------------------------------------------
def check_heat_exact(Nx=64, Nt=16, seed=1):
    """Spectral exponential Euler for u_t = u_xx on [0, 2 pi) is exact in time:
    u(x, t) = sum_k e^{-k^2 t}(a_k cos kx + b_k sin kx)/k^2, evaluated directly."""
    sp = O.Spec("periodic", (Nx,), (2 * math.pi,), 1.0, 0.0, "none", 1.0 / Nt, Nt, 1e-2, 1)
    rng = np.random.default_rng(seed)
    ak, bk = rng.standard_normal(16), rng.standard_normal(16)
    x = np.arange(Nx) * 2 * math.pi / Nx
    def exact(t):
        return sum(math.exp(-k * k * t) * (ak[k - 1] * np.cos(k * x) + bk[k - 1] * np.sin(k * x)) / k**2
                   for k in range(1, 17))
    U = O.sequential_solve(sp, exact(0.0))
    Ue = np.array([exact(n * sp.dt) for n in range(Nt + 1)])
    return O.rel_error(U[1:], Ue[1:])


def check_richardson_closed_form(k_mode=3, iters=4, Nx=16, Nt=8, alpha=0.2):
    """First-order Richardson from zero on u0 = cos(k x): the k-th iterate is
    (1 - (-q)^k) E^n u0 with E = e^{dt mu}, q = alpha E^Nt/(1 - alpha E^Nt)
    (from the error recursion of Sec. 2, Eqs. (2.5)-(2.6))."""
    sp = O.Spec("periodic", (Nx,), (2 * math.pi,), 0.05, 0.02, "none", 0.1, Nt, alpha, 1)
    x = np.arange(Nx) * 2 * math.pi / Nx
    u0 = np.cos(k_mode * x)
    res = O.richardson(sp, u0, max_iter=iters, keep_iterates=True)
    mu = -0.05 * k_mode**2 - 0.02
    E = math.exp(sp.dt * mu)
    q = alpha * E**Nt / (1 - alpha * E**Nt)
    worst = 0.0
    for k, V in enumerate(res.iterates, start=1):
        want = np.array([(1 - (-q) ** k) * E**n * u0 for n in range(1, Nt + 1)])
        worst = max(worst, np.abs(V - want).max())
    return worst


def logistic_exact(u0, t):
    """Exact solution of u' = u - u^3."""
    return u0 * math.exp(t) / math.sqrt(1 - u0**2 + u0**2 * math.exp(2 * t))


def check_nonlinear_order(order, c0=0.4, T=0.5):
    """IF-BDF-s on a spatially constant Allen-Cahn state reduces to BDF-s for
    u' = u - u^3 (A acts as 1 on constants when c = 0).  Returns the observed
    convergence order from dt = T/40 -> T/80 (must be ~ s)."""
    errs = []
    for Nt in (40, 80):
        sp = O.Spec("periodic", (4,), (1.0,), 1e-3, 0.0, "allen_cahn", T / Nt, Nt, 1e-3, order)
        start = np.array([np.full(sp.n, logistic_exact(c0, n * sp.dt)) for n in range(order)])
        U = O.sequential_solve(sp, np.full(sp.n, c0), U_start=start)
        errs.append(abs(U[-1, 0] - logistic_exact(c0, T)))
    return math.log2(errs[0] / errs[1])


def check_forced_order(order, k=2, T=0.5):
    """Linear heat with source e^{-t} cos(kx) on [0, 2pi): the exact Fourier
    coefficient is y(t) = e^{mu t} y0 + (e^{mu t} - e^{-t})/(mu + 1).  Returns
    the observed convergence order of the scheme (must be ~ s)."""
    errs = []
    a = 0.05
    mu = -a * k * k
    for Nt in (40, 80):
        sp = O.Spec("periodic", (8,), (2 * math.pi,), a, 0.0, "none", T / Nt, Nt, 1e-3, order)
        x = np.arange(8) * 2 * math.pi / 8
        f = np.array([math.exp(-(n + 1) * sp.dt) * np.cos(k * x) for n in range(Nt)])
        def y_of(t):
            return math.exp(mu * t) + (math.exp(mu * t) - math.exp(-t)) / (mu + 1.0)
        start = np.array([y_of(n * sp.dt) * np.cos(k * x) for n in range(order)])
        U = O.sequential_solve(sp, np.cos(k * x), f, U_start=start)
        y = y_of(T)
        errs.append(abs(U[-1] @ np.cos(k * x) / 4.0 - y))
    return math.log2(errs[0] / errs[1])


def check_dirichlet_single_mode(order=2, n=(6, 5), p=(2, 3), Nt=10):
    """A grid sine mode is an exact eigenvector of the 5-point Laplacian with
    eigenvalue -(4a/h^2) sum_d sin^2(p_d pi h_d/2) - c; with the source
    e^{-t} times that mode the whole solution stays on it.  Compares with the
    scalar BDF-s recursion for the mode amplitude."""
    a, c, dt = 0.7, 0.2, 0.01
    sp = O.Spec("dirichlet", n, (1.0, 1.0), a, c, "none", dt, Nt, 1e-3, order)
    xs = [np.arange(1, m + 1) / (m + 1) for m in n]
    X, Y = np.meshgrid(*xs, indexing="ij")
    mode = np.sin(p[0] * np.pi * X) * np.sin(p[1] * np.pi * Y)
    lam = -c
    for m, pd in zip(n, p):
        h = 1.0 / (m + 1)
        lam -= a * (4.0 / h**2) * math.sin(pd * math.pi * h / 2) ** 2
    E = math.exp(dt * lam)
    f = np.array([math.exp(-(k + 1) * dt) * mode for k in range(Nt)])
    U = O.sequential_solve(sp, mode, f)
    y = [1.0]
    for m in range(1, Nt + 1):
        q = min(m, order)
        aa, bb = O.bdf_coefficients(q)
        y.append(sum(float(aa[j - 1]) * E**j * y[m - j] for j in range(1, q + 1))
                 + float(bb) * dt * math.exp(-m * dt))
    want = np.array([yy * mode for yy in y])
    return np.abs(U - want).max()


# --- convergence theory ---------------------------------------------------
def check_thm21_contraction(Nx=16, Nt=12, alpha=0.05, iters=5):
    """Ratio of successive errors max_n ||e_n^k|| must not exceed the factor
    |alpha| e^{lambda_max T}/(1 - |alpha| e^{lambda_max T}) of Theorem 2.1;
    returns (max observed ratio) / (bound)."""
    sp = O.Spec("dirichlet", (Nx,), (1.0,), 0.02, 0.5, "none", 0.05, Nt, alpha, 1)
    u0 = np.random.default_rng(5).standard_normal(sp.n)
    ref = O.sequential_solve(sp, u0)[1:]
    res = O.richardson(sp, u0, max_iter=iters, keep_iterates=True)
    errs = [np.sqrt(((ref) ** 2).reshape(Nt, -1).sum(1)).max()]
    for V in res.iterates:
        errs.append(np.sqrt(((V - ref) ** 2).reshape(Nt, -1).sum(1)).max())
    lam_max = O.spatial_eigenvalues(sp).max()
    T = sp.dt * Nt
    bound = alpha * math.exp(lam_max * T) / (1 - alpha * math.exp(lam_max * T))
    ratios = [errs[k] / errs[k - 1] for k in range(1, len(errs))]
    return max(ratios) / bound


def check_gmres_terminates(sp, seed=6):
    """Number of GMRES iterations to reach 1e-12 (Theorem 3.3: <= Nx + 1 for
    s = 1; Theorem 4.3: <= 2 Nx + 1 for s = 2)."""
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    res = O.gmres(sp, u0, f, tol=1e-12, restart=200, max_iter=200)
    return res.iterations, res


def check_gmres_elman(sp, seed=7):
    """max_k ||r_k|| / ((4 alpha (1 - alpha))^{k/2} ||r_0||) for the
    preconditioned GMRES residuals (Theorem 3.14); must be <= 1."""
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(sp.n)
    res = O.gmres(sp, u0, None, tol=1e-14, restart=50, max_iter=30)
    q = 4 * sp.alpha * (1 - sp.alpha)
    return max(h / q ** (k / 2) for k, h in enumerate(res.history))


def check_bicgstab_minimal_polynomial(eigs=(2.0, 2.0, 5.0, 5.0, 5.0, -1.5), seed=8, rotate=True):
    """BiCGStab on A = Q diag(eigs) Q^{-1}: with d distinct eigenvalues the
    BiCG residual polynomial annihilates r_0 after d steps (exact arithmetic),
    so BiCGStab's history must reach rounding level by iteration d.  Returns
    (history, d, error of x vs the direct solve)."""
    rng = np.random.default_rng(seed)
    n = len(eigs)
    Q = np.eye(n) + (0.3 * rng.standard_normal((n, n)) if rotate else 0.0)
    A = Q @ np.diag(eigs) @ np.linalg.inv(Q)
    b = rng.standard_normal(n)
    x, hist = O.bicgstab_solve(lambda v: A @ v, b, 1e-300, len(set(eigs)))
    err = float(np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(np.linalg.solve(A, b)))
    return hist, len(set(eigs)), err


def check_bicgstab_reaches_sequential(sp, seed=9):
    """Relative error of the oracle's BiCGStab solution vs sequential stepping."""
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(sp.n)
    f = rng.standard_normal((sp.Nt,) + sp.n)
    ref = O.sequential_solve(sp, u0, f)
    res = O.bicgstab(sp, u0, f, tol=1e-13)
    return O.rel_error(res.U[1:], ref[1:]), res


def check_precond_shift_vs_dense(sp, shift=0.3, seed=11):
    """(P_alpha - shift I)^{-1} by the three steps vs the dense LU solve."""
    r = rng_field(sp, seed, (sp.Ns,))
    ref = O.dense_precond_apply(sp, r, shift)
    return np.abs(O.precond_apply(sp, r, shift) - ref).max() / np.abs(ref).max()


def check_mean_jacobian_contraction(order=1, c0=0.1, iters=4):
    """Allen-Cahn from a constant state u_0 = c0 (N'(u_0) = 1 - 3 c0^2 ~ 1 is the
    Jacobian at t = 0 everywhere): observed contraction of the lagged iteration
    and of the mean-Jacobian (inexact Newton) iteration, (rho_lagged, rho_newton)."""
    sp = O.Spec("periodic", (8,), (1.0,), 0.01, 0.0, "allen_cahn", 0.05, 24, 1e-3, order)
    u0 = np.full(sp.n, c0) + 1e-3 * np.cos(2 * np.pi * np.arange(8) / 8)
    ref = O.sequential_solve(sp, u0)[1:]
    out = []
    for jac in ("lagged", "mean_u0"):
        errs = []
        for k in range(1, iters + 1):
            U = O.richardson(sp, u0, None, max_iter=k, jacobian=jac).U[1:]
            errs.append(O.rel_error(U, ref))
        out.append(max(errs[k] / errs[k - 1] for k in range(1, len(errs))))
    return tuple(out)


# --- advection-diffusion (periodic) ----------------------------------------
def adv_spec(n=(8,), length=None, b=(0.7,), order=1, Nt=9, nonlin="none", a=0.3, c=0.1, alpha=0.05, dt=0.05):
    if length is None:
        length = tuple(2 * math.pi for _ in n)
    return O.Spec("periodic", tuple(n), tuple(length), a, c, nonlin, dt, Nt, alpha, order, tuple(b))


def check_advection_exact(Nx=64, Nt=16, b=2.0, a=0.1, seed=2):
    """u_t = a u_xx - b u_x on [0, 2 pi): u = sum_k e^{-a k^2 t} (a_k cos k(x - bt)
    + b_k sin k(x - bt))/k^2 exactly; spectral exponential Euler is exact in time."""
    sp = O.Spec("periodic", (Nx,), (2 * math.pi,), a, 0.0, "none", 1.0 / Nt, Nt, 1e-2, 1, (b,))
    rng = np.random.default_rng(seed)
    ak, bk = rng.standard_normal(16), rng.standard_normal(16)
    x = np.arange(Nx) * 2 * math.pi / Nx

    def exact(t):
        return sum(math.exp(-a * k * k * t) * (ak[k - 1] * np.cos(k * (x - b * t)) + bk[k - 1] * np.sin(k * (x - b * t)))
                   / k**2 for k in range(1, 17))
    U = O.sequential_solve(sp, exact(0.0))
    Ue = np.array([exact(n * sp.dt) for n in range(Nt + 1)])
    return O.rel_error(U[1:], Ue[1:])


# --- initial iterate --------------------------------------------------------
def check_linear_guess_is_homogeneous_solution():
    """Without N and f the scheme's solution is u_n = A^n u_0 (the BDF
    coefficients sum to one), so `linear_guess` must equal sequential stepping
    there, for every order and grid, advection included; returns the worst
    relative difference."""
    worst = 0.0
    cases = [spec("periodic", (12,), a=0.05, c=0.1, Nt=order + 9, order=order, dt=0.03) for order in (1, 2, 6)]
    cases += [spec("dirichlet", (7, 5), a=0.02, c=0.1, Nt=order + 7, order=order, dt=0.05) for order in (1, 3)]
    cases += [O.Spec("periodic", (16,), (1.0,), 0.01, 0.0, "none", 0.02, 10, 0.01, 2, b=(0.7,))]
    for sp in cases:
        u0 = np.random.default_rng(sp.order + sp.Nt).standard_normal(sp.n)
        ref = O.sequential_solve(sp, u0)
        U_start = O.startup_values(sp, u0)
        V = O.linear_guess(sp, U_start)
        worst = max(worst, O.rel_error(V, ref[sp.order:]))
    return worst


# --- ETD1 (phi_1) ------------------------------------------------------------
def etd_spec(bc="periodic", n=(8,), Nt=6, a=0.3, c=0.1, dt=0.05, alpha=0.05):
    sp = spec(bc, n, a=a, c=c, nonlin="allen_cahn", dt=dt, Nt=Nt, alpha=alpha, order=1)
    return O.Spec(sp.bc, sp.n, sp.length, sp.a, sp.c, sp.nonlin, sp.dt, sp.Nt, sp.alpha, sp.order, (), "etd1")


def check_phi1_scalar():
    """phi_1(z) = (e^z - 1)/z against a 40-digit evaluation (decimal), with
    phi_1(0) = 1, over arguments from -700 to 1 including tiny ones."""
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    zs = np.array([-700.0, -50.0, -3.0, -1.0, -1e-3, -1e-9, -1e-300, 0.0, 1e-12, 1e-4, 0.5, 1.0])
    got = O.phi1(zs)
    worst = 0.0
    for z, g in zip(zs, got):
        dz = Decimal(float(z))
        if abs(z) < 1e-20:
            want = 1 + dz / 2          # the series: 1 + z/2 + z^2/6 + ...
        else:
            want = (dz.exp() - 1) / dz
        worst = max(worst, abs(float((Decimal(float(g)) - want) / want)))
    return worst


def check_phi1_vs_dense(sp, seed=12):
    """dt phi_1(dt L_h) u by the eigen-symbol path against the top-right block
    of the dense expm of [[dt L_h, I], [0, 0]]."""
    u = rng_field(sp, seed)
    ref = (O.dense_phi1(sp) @ u.ravel()).reshape(sp.n)
    return np.abs(O.apply_phi1(sp, u) - ref).max() / np.abs(ref).max()


def check_etd1_sequential_vs_dense(sp, seed=13):
    """ETD1 stepping (eigen symbols) against the dense all-at-once system
    R_1 v - (C_0 (x) Phi) N(v) = b solved by Newton with dense expm operators."""
    u0 = 0.6 * np.tanh(rng_field(sp, seed))
    U = O.sequential_solve(sp, u0)
    D = O.dense_solve(sp, u0)
    return np.abs(U - D).max() / np.abs(D).max()


def check_etd1_order(T=0.4, n=16, a=0.05):
    """ETD1 on the semi-discrete 1D periodic Allen-Cahn system against
    scipy's DOP853 at tolerance 1e-12 (dense L_h): the observed convergence
    order from Nt = 40 -> 80 (must be ~ 1)."""
    import scipy.integrate
    x = np.arange(n) * 2 * math.pi / n
    u0 = 0.5 * np.sin(x) + 0.2 * np.cos(2 * x)
    base = O.Spec("periodic", (n,), (2 * math.pi,), a, 0.0, "allen_cahn", T / 40, 40, 1e-3, 1, (), "etd1")
    L = O.dense_Lh(base)
    sol = scipy.integrate.solve_ivp(lambda t, u: L @ u + u - u**3, (0.0, T), u0, method="DOP853",
                                    rtol=1e-12, atol=1e-14)
    ref = sol.y[:, -1]
    errs = []
    for Nt in (40, 80):
        sp = O.Spec("periodic", (n,), (2 * math.pi,), a, 0.0, "allen_cahn", T / Nt, Nt, 1e-3, 1, (), "etd1")
        U = O.sequential_solve(sp, u0)
        errs.append(np.abs(U[-1] - ref).max())
    return math.log2(errs[0] / errs[1])


def check_etd1_richardson_reaches_sequential(sp, seed=14, iters=80):
    """The lagged Exp-ParaDiag fixed point of the ETD1 system (residual with
    N of the previous slice) reaches the sequential ETD1 solution."""
    u0 = 0.6 * np.tanh(rng_field(sp, seed))
    ref = O.sequential_solve(sp, u0)
    res = O.richardson(sp, u0, None, max_iter=iters, tol=1e-15)
    return O.rel_error(res.U[1:], ref[1:])


# --- complex states: the Schrodinger equation of Sec. 7 --------------------
def se_spec(bc="dirichlet", n=(7,), a=1j, c=2j, Nt=8, order=1, alpha=0.05, dt=0.05, length=None):
    if length is None:
        length = tuple(2 * math.pi if bc == "periodic" else 1.0 for _ in n)
    return O.Spec(bc, tuple(n), tuple(length), a, c, "none", dt, Nt, alpha, order, complex_state=True)


def rng_complex(sp, seed, lead=()):
    rng = np.random.default_rng(seed)
    shape = tuple(lead) + sp.n
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def check_complex_A_vs_dense(sp, seed=20):
    """A^j u for a complex state and complex a, c: eigen-symbol path against
    the dense expm of the explicit complex L_h (j = 1..3)."""
    A = O.dense_A(sp)
    u = rng_complex(sp, seed)
    worst, Aj = 0.0, np.eye(A.shape[0], dtype=complex)
    for j in range(1, 4):
        Aj = Aj @ A
        ref = (Aj @ u.ravel()).reshape(sp.n)
        worst = max(worst, np.abs(O.apply_A_power(sp, u, j) - ref).max() / np.abs(ref).max())
    return worst


def check_complex_precond_vs_dense(sp, seed=21):
    r = rng_complex(sp, seed, (sp.Ns,))
    ref = O.dense_precond_apply(sp, r)
    return np.abs(O.precond_apply(sp, r) - ref).max() / np.abs(ref).max()


def check_complex_sequential_vs_dense(sp, seed=22):
    u0 = rng_complex(sp, seed)
    f = rng_complex(sp, seed + 1, (sp.Nt,))
    return O.rel_error(O.sequential_solve(sp, u0, f)[1:], O.dense_solve(sp, u0, f)[1:])


def check_schrodinger_sine_mode(n=15, Nt=12, dt=0.01, c=2j):
    """u_0 = sin(pi x) is the first eigenvector of the 3-point Dirichlet
    Laplacian (eigenvalue -(4/h^2) sin^2(pi h/2)); with a = i the first-order
    scheme gives u_n = exp(n dt (i lambda_1 - c)) u_0 exactly.  Max deviation."""
    sp = se_spec("dirichlet", (n,), 1j, c, Nt, 1, dt=dt)
    x = np.arange(1, n + 1) / (n + 1)
    u0 = np.sin(np.pi * x).astype(complex)
    h = 1.0 / (n + 1)
    lam1 = -(4.0 / h**2) * math.sin(math.pi * h / 2) ** 2
    mu = 1j * lam1 - c
    want = np.array([np.exp(k * dt * mu) * u0 for k in range(Nt + 1)])
    return np.abs(O.sequential_solve(sp, u0) - want).max()


def check_unitary_norm(sp, seed=23):
    """Purely imaginary a and c make A = exp(dt L_h) unitary, and every BDF-s
    step of a homogeneous problem reproduces u_n = A^n u_0 (the a_j sum to 1);
    max_n | ||u_n|| / ||u_0|| - 1 |."""
    u0 = rng_complex(sp, seed)
    U = O.sequential_solve(sp, u0)
    nrm = np.sqrt((np.abs(U.reshape(U.shape[0], -1)) ** 2).sum(1))
    return float(np.abs(nrm / nrm[0] - 1.0).max())


def schrodinger_gmres_errors(p, iters):
    """Errors (Sec. 7's norm) vs sequential stepping after k = 1..iters GMRES
    iterations on a Schrodinger workload."""
    from paper_2603_04350_gb300 import inputs as I
    sp = O.spec_of(p)
    u0, f = I.make_inputs(p)
    seq = O.sequential_solve(sp, u0, f)
    return [O.rel_error(O.gmres(sp, u0, f, tol=0.0, restart=20, max_iter=k).U[1:], seq[1:])
            for k in range(1, iters + 1)]


def check_complex_gmres_vs_dense(sp, seed=24):
    """Complex GMRES solution vs the dense LU solution."""
    u0 = rng_complex(sp, seed)
    f = rng_complex(sp, seed + 1, (sp.Nt,))
    res = O.gmres(sp, u0, f, tol=1e-13, restart=50, max_iter=100)
    return O.rel_error(res.U[1:], O.dense_solve(sp, u0, f)[1:]), res


def check_complex_bicgstab_vs_dense(sp, seed=25):
    u0 = rng_complex(sp, seed)
    f = rng_complex(sp, seed + 1, (sp.Nt,))
    res = O.bicgstab(sp, u0, f, tol=1e-13, max_iter=100)
    return O.rel_error(res.U[1:], O.dense_solve(sp, u0, f)[1:]), res


# --- Neumann grids (DCT-II eigenbasis; the Allen-Cahn experiment of Sec. 7) --
def neu_spec(n=(8,), a=0.3, c=0.1, nonlin="none", Nt=9, order=1, alpha=0.05, dt=0.05):
    return O.Spec("neumann", tuple(n), tuple(1.0 for _ in n), a, c, nonlin, dt, Nt, alpha, order)


def check_neumann_mass(n=(12,), Nt=10, order=2):
    """With c = 0 and no source the mirrored boundary lets nothing out: the
    cell sum sum_j u_n,j (the k = 0 mode, symbol 0) is conserved.  Max
    relative drift."""
    sp = neu_spec(n, a=0.7, c=0.0, Nt=Nt, order=order, dt=0.01)
    u0 = np.random.default_rng(30).uniform(-1, 1, sp.n) + 0.3
    U = O.sequential_solve(sp, u0)
    m = U.reshape(U.shape[0], -1).sum(1)
    return float(np.abs(m / m[0] - 1.0).max())


def check_neumann_cosine_mode(n=16, k=2, Nt=8, a=0.7, c=0.2, dt=0.01):
    """cos(k pi x_j) at the cell centres is an eigenvector of the Neumann
    3-point Laplacian with eigenvalue -(4/h^2) sin^2(k pi/(2n)); the first-order
    scheme multiplies it by exp(dt mu) per step.  Max deviation."""
    sp = neu_spec((n,), a, c, Nt=Nt, order=1, dt=dt)
    x = (np.arange(n) + 0.5) / n
    u0 = np.cos(k * np.pi * x)
    h = 1.0 / n
    mu = -a * (4.0 / h**2) * math.sin(k * math.pi / (2 * n)) ** 2 - c
    want = np.array([math.exp(j * dt * mu) * u0 for j in range(Nt + 1)])
    return np.abs(O.sequential_solve(sp, u0) - want).max()


def neumann_allen_cahn_errors(order, n=256, T=0.1, steps=(25, 50, 100, 200), eps=0.01):
    """The Neumann Allen-Cahn problem of Sec. 7: u_t = eps^2 u_xx - (u^3 - u)
    + s_f on (0, 1), du/dn = 0, eps = 0.01, the source chosen so that
    u = 0.5 e^{-t} cos(2 pi x) is the exact solution
    (s_f = u (4 pi^2 eps^2 - 2) + u^3); Sec. 7's error of the sequential
    IF-BDF-s solution at each step count."""
    out = []
    for Nt in steps:
        dt = T / Nt
        sp = O.Spec("neumann", (n,), (1.0,), eps**2, 0.0, "allen_cahn", dt, Nt, 1e-3, order)
        x = (np.arange(n) + 0.5) / n

        def ue(t):
            return 0.5 * np.exp(-t) * np.cos(2 * np.pi * x)
        f = np.array([ue((k + 1) * dt) * (4 * np.pi**2 * eps**2 - 2) + ue((k + 1) * dt) ** 3
                      for k in range(Nt)])
        U = O.sequential_solve(sp, ue(0.0), f)
        ex = np.array([ue(k * dt) for k in range(Nt + 1)])
        out.append(O.rel_error(U[1:], ex[1:]))
    return out


def check_wraparound_identity(bc="dirichlet", n=(9,), order=2, Nt=12, alpha=1e-2, seed=0):
    """R_s and the alpha-circulant preconditioner P_alpha = R_s^alpha differ only
    in the wrap-around entries: R_s - R_s^alpha = alpha W_s with
    (W_s v)_n = sum_{j = n+1..s} a_j A^j v_{n-j+Ns}, nonzero in the first s slices
    (C_{j-1}^alpha - C_{j-1} is alpha in the top-right corner, Eq. (2.4) and
    reading 1).  Hence P_alpha^{-1} R_s v = v + alpha P_alpha^{-1} (W_s v) for
    s < Ns: checked through the oracle's three-step preconditioner, and W_s
    against the dense R_s - R_s^alpha.  Returns the larger relative error."""
    sp = O.Spec(bc, tuple(n), tuple(1.0 for _ in n), 0.02, 0.1, "none", 0.01, Nt, alpha, order)
    Ns = sp.Ns
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((Ns,) + sp.n)
    a, _ = O.bdf_float(order)
    W = np.zeros_like(V)
    for i in range(min(order, Ns)):
        for j in range(i + 1, order + 1):
            if i - j + Ns >= 0:
                W[i] += a[j - 1] * O.apply_A_power(sp, V[i - j + Ns], j)
    lhs = O.precond_apply(sp, O.apply_R(sp, V))
    rhs = V + alpha * O.precond_apply(sp, W)
    e1 = np.abs(lhs - rhs).max() / np.abs(lhs).max()
    D = (O.dense_R(sp, 0.0) - O.dense_R(sp, alpha)) @ V.reshape(-1)
    e2 = np.abs(D - alpha * W.reshape(-1)).max() / np.abs(alpha * W).max()
    return max(e1, e2)


def check_dst_mirror_fold(n=12, seed=0):
    """The orthonormal DST-I S (L_h's Dirichlet eigenvectors, Sec. 3.1) satisfies
    S[j][n-1-k] = (-1)^j S[j][k], so for even n output j of a row x is
    sum_{k < n/2} S[j][k] (x_k + (-1)^j x_{n-1-k}).  S is taken from the oracle's
    eigenbasis transform applied to unit vectors; returns the larger of the
    symmetry's and the folded product's errors."""
    sp = O.Spec("dirichlet", (n,), (1.0,), 0.02, 0.1, "none", 0.01, 4, 0.01, 1)
    S = np.array([O.to_eigen(sp, e) for e in np.eye(n)]).T  # column k = transform of e_k
    j = np.arange(n)[:, None]
    e1 = np.abs(S[:, ::-1] - ((-1.0) ** j) * S).max()
    x = np.random.default_rng(seed).standard_normal(n)
    h = n // 2
    u, v = x[:h] + x[::-1][:h], x[:h] - x[::-1][:h]
    y = np.empty(n)
    y[0::2] = S[0::2, :h] @ u
    y[1::2] = S[1::2, :h] @ v
    e2 = np.abs(y - S @ x).max() / np.abs(S @ x).max()
    return max(e1, e2)
