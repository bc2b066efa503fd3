"""CPU float64 oracle for Exp-ParaDiag -- TEST INFRASTRUCTURE, not product code.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg
may import this module.  It shares no code with the CUDA path and never imports
the product package; inputs reach it as plain numpy arrays.

It is a plain, slow, obviously-correct numpy restatement (float64 throughout) of
what Garai & Chamakuri, "Exp-ParaDiag: Time-Parallel Exponential Integrators for
Parabolic PDEs" (arXiv 2603.04350) computes:

  * the exponential BDF-s schemes u_n = sum_j a_j A^j u_{n-j}, A = exp(dt L_h)
    (Eq. (4.1), Sec. 5 Eqs. (5.1), (5.3), (5.5), (5.7)), with the
    integrating-factor nonlinear term of Eq. (6.1) and a source term;
  * the all-at-once systems Q u = f / R_s v = f_s (Eqs. (3.1), (4.2), Sec. 5)
    and their alpha-circulant preconditioners (Eqs. (3.2), (4.4), Sec. 5);
  * the three-step preconditioner solve (Eq. (3.3), Eq. (4.5));
  * the preconditioned Richardson iteration (Eq. (3.2), (4.4)) and its lagged
    nonlinear form (Eqs. (7.3)-(7.4));
  * left-preconditioned GMRES (Sec. 3.2, Theorem 3.3) and BiCGStab;
  * periodic (spectral), Dirichlet (DST-I) and Neumann (cell-centred, DCT-II)
    grids, the Neumann one for the Allen-Cahn experiment of Sec. 7;
  * complex states for complex a and c, the Schrodinger equation of Sec. 7
    (a = i, c = 2i or 200i): complex arithmetic throughout, GMRES with the
    Hermitian inner product and complex Givens rotations;
  * dense brute-force versions of all of the above for tiny sizes (explicit
    L_h, scipy's expm, explicit C_j^alpha matrices, LU solves).

Readings taken where the paper is silent: GMRES on a complex state is complex
GMRES (the paper's Schrodinger runs converge in one and three iterations,
which real GMRES on the real and imaginary parts does not reproduce); the source f enters row n as beta_s*dt*f(t_n) and the nonlinear term as
beta_s*dt*N(u_n) (implicit, integrating factor); the startup values
u_1..u_{s-1} come from the IF-BDF_j ramp j = 1..s-1; C_j^alpha = (C_0^alpha)^(j+1)
(the printed entry lists of Sec. 5 are garbled); the periodic L_h is the
spectral Laplacian with the Nyquist mode's symbol -a*(pi*n/L)^2; the Neumann
L_h is the 3-point Laplacian on cell centres with mirrored ghost values (the
paper names the boundary condition, not its discretisation).

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, the paper's printed coefficients and spectra, and dense
brute force; nothing is "parity unpinned".
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass
from fractions import Fraction
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.fft
import scipy.linalg

PERIODIC = "periodic"
DIRICHLET = "dirichlet"
NEUMANN = "neumann"


# ---------------------------------------------------------------------------
# Problem description (plain data; the oracle does not import the product).
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Spec:
    bc: str                      # "periodic" | "dirichlet" | "neumann"
    n: Tuple[int, ...]           # grid points per dimension
    length: Tuple[float, ...]    # domain length per dimension
    a: complex                   # L = a*Lap - c   (Eq. (1.2)); a = i, c = 2i: Schrodinger (Sec. 7)
    c: complex
    nonlin: str                  # "none" | "allen_cahn"
    dt: float
    Nt: int
    alpha: float
    order: int                   # s in 1..6
    b: Tuple[float, ...] = ()    # advection velocity: L = a*Lap - b.grad - c (periodic only)
    nl_form: str = "if"          # "if" (integrating factor, Eq. (6.1)) | "etd1" (see etd1_step)
    complex_state: bool = False  # u, f and the solution are complex (Schrodinger-type L, Sec. 7)

    @property
    def ndim(self):
        return len(self.n)

    @property
    def Ns(self):
        return self.Nt - self.order + 1


def spec_of(p) -> Spec:
    """Build a Spec from any object with the same attribute names."""
    return Spec(p.bc, tuple(p.n), tuple(p.length), p.a, p.c, p.nonlin, p.dt, p.Nt,
                p.alpha, p.order, tuple(getattr(p, "b", ()) or ()), getattr(p, "nl_form", "if"),
                bool(getattr(p, "complex_state", False)))


def state_dtype(sp: Spec):
    """float64 for a real state; complex128 when the state is complex, as for
    the Schrodinger equation u_t = i Lap u - c u of Sec. 7 (a = i, c = 2i or
    200i), whose solution is complex even from a real u_0."""
    if not sp.complex_state and (np.imag(sp.a) != 0 or np.imag(sp.c) != 0):
        raise ValueError("a complex a or c needs complex_state=True")
    if sp.complex_state and sp.nonlin != "none":
        raise ValueError("a complex state is defined for linear problems only")
    return np.complex128 if sp.complex_state else np.float64


def has_advection(sp: Spec) -> bool:
    return any(v != 0.0 for v in sp.b)


# ---------------------------------------------------------------------------
# BDF coefficients (Eq. (4.1), Eqs. (5.1), (5.3), (5.5), (5.7)).
# ---------------------------------------------------------------------------
def bdf_coefficients(s: int) -> Tuple[List[Fraction], Fraction]:
    """Exact a_1..a_s and beta_s of BDF-s from its defining difference form
    sum_{i=1..s} (1/i) nabla^i u_n = dt f_n, i.e. the polynomial
    sum_i (1/i)(1 - z)^i = c_0 + c_1 z + ... normalised to u_n - sum_j a_j u_{n-j}
    = beta dt f_n.  The paper prints the resulting a_j for s = 2..6."""
    if not 1 <= s <= 6:
        raise ValueError("order must be 1..6")
    c = [Fraction(0)] * (s + 1)
    for i in range(1, s + 1):
        for j in range(i + 1):
            c[j] += Fraction(1, i) * math.comb(i, j) * (-1) ** j
    beta = 1 / c[0]
    a = [-c[j] / c[0] for j in range(1, s + 1)]
    return a, beta


def bdf_float(s: int):
    a, beta = bdf_coefficients(s)
    return np.array([float(x) for x in a]), float(beta)


# ---------------------------------------------------------------------------
# Spatial operator L_h = a*Delta_h - c and its eigenbasis (Sec. 2, after Eq. (2.7)).
# ---------------------------------------------------------------------------
def spatial_eigenvalues(sp: Spec) -> np.ndarray:
    """Eigenvalues mu of L_h laid out like the oracle's eigen-coefficients.

    Periodic: spectral Laplacian, mu = -a*sum_d (2*pi*k_d/L_d)^2 - c with k_d in
    numpy FFT order (the Nyquist index carries (pi*n/L)^2).
    Dirichlet: 3-point (1D) / 5-point (2D) finite differences on n interior
    points, h = L/(n+1): mu = -a*sum_d (4/h^2) sin^2(pi k_d h/(2 L_d)) - c,
    k_d = 1..n, eigenvectors sin(pi k_d x/L_d) (the DST-I basis).
    Neumann (the Allen-Cahn experiment of Sec. 7 with du/dn = 0): the same
    finite differences on the n cell centres x_j = (j - 1/2) h, h = L/n, with
    the boundary condition imposed by mirroring (u_0 = u_1, u_{n+1} = u_n):
    mu = -a*sum_d (4/h^2) sin^2(pi k_d/(2 n_d)) - c, k_d = 0..n-1,
    eigenvectors cos(pi k_d (j - 1/2)/n_d) (the DCT-II basis).
    Advection (periodic, the advection-diffusion operator of Sec. 7 and
    Remark 3.7): the spectral first derivative adds -i sum_d b_d (2 pi k_d/L_d)
    with the Nyquist wavenumber's first-derivative symbol 0 (so real fields
    stay real); mu is then complex with mu(-k) = conj(mu(k))."""
    parts, adv = [], []
    for d, (n, L) in enumerate(zip(sp.n, sp.length)):
        if sp.bc == PERIODIC:
            k = np.fft.fftfreq(n, 1.0 / n)
            parts.append(-(2.0 * np.pi * k / L) ** 2)
            k1 = k.copy()
            if n % 2 == 0:
                k1[n // 2] = 0.0
            adv.append(2.0 * np.pi * k1 / L * (sp.b[d] if d < len(sp.b) else 0.0))
        elif sp.bc == NEUMANN:
            h = L / n
            k = np.arange(n)
            parts.append(-(4.0 / h**2) * np.sin(np.pi * k / (2.0 * n)) ** 2)
        else:
            h = L / (n + 1)
            k = np.arange(1, n + 1)
            parts.append(-(4.0 / h**2) * np.sin(np.pi * k * h / (2.0 * L)) ** 2)
    if has_advection(sp) and sp.bc != PERIODIC:
        raise ValueError("advection needs a periodic grid")
    grids = np.meshgrid(*parts, indexing="ij")
    mu = sp.a * sum(grids) - sp.c
    if has_advection(sp):
        mu = mu - 1j * sum(np.meshgrid(*adv, indexing="ij"))
    return mu


def _axes(sp: Spec, x: np.ndarray):
    return tuple(range(x.ndim - sp.ndim, x.ndim))


def to_eigen(sp: Spec, u: np.ndarray) -> np.ndarray:
    """Coefficients of u in L_h's eigenbasis (last ndim axes): unnormalised
    DFT for periodic grids, orthonormal DST-I for Dirichlet grids, orthonormal
    DCT-II for Neumann grids."""
    ax = _axes(sp, u)
    if sp.bc == PERIODIC:
        return np.fft.fftn(u, axes=ax)
    if sp.bc == NEUMANN:
        if np.iscomplexobj(u):
            return (scipy.fft.dctn(u.real, type=2, axes=ax, norm="ortho")
                    + 1j * scipy.fft.dctn(u.imag, type=2, axes=ax, norm="ortho"))
        return scipy.fft.dctn(u, type=2, axes=ax, norm="ortho")
    if np.iscomplexobj(u):
        return (scipy.fft.dstn(u.real, type=1, axes=ax, norm="ortho")
                + 1j * scipy.fft.dstn(u.imag, type=1, axes=ax, norm="ortho"))
    return scipy.fft.dstn(u, type=1, axes=ax, norm="ortho")


def from_eigen(sp: Spec, uh: np.ndarray) -> np.ndarray:
    """Inverse of to_eigen (complex in, complex out for periodic grids)."""
    ax = _axes(sp, uh)
    if sp.bc == PERIODIC:
        return np.fft.ifftn(uh, axes=ax)
    if sp.bc == NEUMANN:
        if np.iscomplexobj(uh):
            return (scipy.fft.idctn(uh.real, type=2, axes=ax, norm="ortho")
                    + 1j * scipy.fft.idctn(uh.imag, type=2, axes=ax, norm="ortho"))
        return scipy.fft.idctn(uh, type=2, axes=ax, norm="ortho")
    if np.iscomplexobj(uh):
        return (scipy.fft.idstn(uh.real, type=1, axes=ax, norm="ortho")
                + 1j * scipy.fft.idstn(uh.imag, type=1, axes=ax, norm="ortho"))
    return scipy.fft.idstn(uh, type=1, axes=ax, norm="ortho")


def apply_A_power(sp: Spec, u: np.ndarray, j: int) -> np.ndarray:
    """A^j u with A = exp(dt L_h) (Eq. (2.2)), applied in L_h's eigenbasis."""
    mu = spatial_eigenvalues(sp)
    out = from_eigen(sp, np.exp(j * sp.dt * mu) * to_eigen(sp, u))
    return out if (np.iscomplexobj(u) or sp.complex_state) else out.real


# ---------------------------------------------------------------------------
# phi_1 and the first-order exponential time differencing (ETD1) step.
# Sec. 6 names an ETD-based treatment of the nonlinear term as the
# alternative to the integrating factor it develops; ETD1 is its first-order
# member: u_n = A u_{n-1} + dt phi_1(dt L_h) N(u_{n-1}), phi_1(z) = (e^z - 1)/z.
# ---------------------------------------------------------------------------
def phi1(z: np.ndarray) -> np.ndarray:
    """phi_1(z) = (e^z - 1)/z, phi_1(0) = 1; expm1 keeps small |z| accurate."""
    z = np.asarray(z)
    out = np.ones(z.shape, dtype=np.result_type(z, np.float64))
    nz = z != 0
    out[nz] = np.expm1(z[nz]) / z[nz]
    return out


def apply_phi1(sp: Spec, u: np.ndarray) -> np.ndarray:
    """dt phi_1(dt L_h) u, applied in L_h's eigenbasis."""
    mu = spatial_eigenvalues(sp)
    out = from_eigen(sp, sp.dt * phi1(sp.dt * mu) * to_eigen(sp, u))
    return out if np.iscomplexobj(u) else out.real


def etd1_step(sp: Spec, u_prev: np.ndarray) -> np.ndarray:
    """u_n = A u_{n-1} + dt phi_1(dt L_h) N(u_{n-1}) (explicit in N)."""
    return apply_A_power(sp, u_prev, 1) + apply_phi1(sp, nonlinearity(sp, u_prev))


def _check_etd1(sp: Spec, f) -> None:
    if sp.order != 1:
        raise ValueError("ETD1 is a first-order scheme (order 1)")
    if f is not None:
        raise ValueError("the ETD1 form takes no source term")


# ---------------------------------------------------------------------------
# Nonlinearity and the pointwise implicit solve of the IF scheme (Eq. (6.1)).
# ---------------------------------------------------------------------------
def nonlinearity(sp: Spec, u: np.ndarray) -> np.ndarray:
    """N(u): zero for linear problems, u - u^3 for Allen-Cahn."""
    if sp.nonlin == "none":
        return np.zeros_like(u)
    if sp.nonlin == "allen_cahn":
        return u - u**3
    raise ValueError(sp.nonlin)


def pointwise_implicit_solve(sp: Spec, w: np.ndarray, bdt: float) -> np.ndarray:
    """Solve u - bdt*N(u) = w pointwise (the implicit IF step of Eq. (6.1)).
    For Allen-Cahn g(u) = u - bdt(u - u^3) - w is strictly increasing when
    bdt < 1, so Newton from u = w converges to the unique root."""
    if sp.nonlin == "none":
        return w.copy()
    if not bdt < 1.0:
        raise ValueError("pointwise solve needs beta*dt < 1")
    u = w.copy()
    for _ in range(60):
        g = u - bdt * (u - u**3) - w
        dg = 1.0 - bdt + 3.0 * bdt * u**2
        du = g / dg
        u = u - du
        if np.max(np.abs(du)) <= 1e-16 * max(1.0, float(np.max(np.abs(u)))):
            break
    return u


# ---------------------------------------------------------------------------
# Sequential time stepping: the exact solution of the all-at-once system.
# ---------------------------------------------------------------------------
def step_rhs(sp: Spec, U: np.ndarray, n: int, q: int, f: Optional[np.ndarray]) -> np.ndarray:
    """w_n = sum_{j=1..q} a_j A^j u_{n-j} + beta_q dt f(t_n) of BDF-q."""
    a, beta = bdf_float(q)
    w = np.zeros(sp.n, dtype=state_dtype(sp))
    for j in range(1, q + 1):
        w += a[j - 1] * apply_A_power(sp, U[n - j], j)
    if f is not None:
        w += beta * sp.dt * f[n - 1]
    return w


def sequential_solve(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None,
                     U_start: Optional[np.ndarray] = None) -> np.ndarray:
    """u_0..u_Nt by sequential exponential BDF stepping, shape (Nt+1, *n).

    Steps n >= s use BDF-s (Eqs. (2.2), (4.1), (5.1), (5.3), (5.5), (5.7)).
    The paper treats u_1..u_{s-1} as given (Eqs. (4.2), (5.2)-(5.8)); they are
    taken from U_start (shape (s, *n), U_start[0] = u0) when supplied, else
    from the ramp that steps u_n with BDF-n.  Each step solves
    u_n - beta dt N(u_n) = sum_j a_j A^j u_{n-j} + beta dt f(t_n)."""
    U = np.zeros((sp.Nt + 1,) + sp.n, dtype=state_dtype(sp))
    U[0] = u0
    if sp.nl_form == "etd1" and sp.nonlin != "none":
        _check_etd1(sp, f)
        for n in range(1, sp.Nt + 1):
            U[n] = etd1_step(sp, U[n - 1])
        return U
    first = 1
    if U_start is not None:
        U[: sp.order] = U_start
        first = sp.order
    for n in range(first, sp.Nt + 1):
        q = min(n, sp.order)
        _, beta = bdf_float(q)
        w = step_rhs(sp, U, n, q, f)
        U[n] = pointwise_implicit_solve(sp, w, beta * sp.dt)
    return U


def startup_values(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None,
                   U_start: Optional[np.ndarray] = None) -> np.ndarray:
    """u_0..u_{s-1}: the given values, or u0 and the sequential ramp."""
    if U_start is not None:
        return np.array(U_start, dtype=state_dtype(sp)).reshape((sp.order,) + sp.n)
    short = dataclasses.replace(sp, Nt=sp.order - 1)
    if sp.order == 1:
        return u0[None].copy()
    return sequential_solve(short, u0, f)


# ---------------------------------------------------------------------------
# The all-at-once system (Eqs. (3.1), (4.2), (5.2), (5.4), (5.6), (5.8)).
# Unknowns v = (u_s, ..., u_Nt): Ns = Nt - s + 1 slices; row i is time n = s+i.
# ---------------------------------------------------------------------------
def rhs_known(sp: Spec, U_start: np.ndarray, f: Optional[np.ndarray]) -> np.ndarray:
    """The known right-hand side f_s: the startup terms a_j A^j u_{n-j} with
    n-j < s (the printed f_2 .. f_6) plus beta_s dt f(t_n)."""
    s = sp.order
    a, beta = bdf_float(s)
    b = np.zeros((sp.Ns,) + sp.n, dtype=state_dtype(sp))
    for i in range(sp.Ns):
        n = s + i
        if f is not None:
            b[i] += beta * sp.dt * f[n - 1]
        for j in range(1, s + 1):
            if n - j < s:
                b[i] += a[j - 1] * apply_A_power(sp, U_start[n - j], j)
    if is_etd1(sp):
        # ETD1: row 0 also carries the known dt phi_1(dt L_h) N(u_0)
        _check_etd1(sp, f)
        b[0] += apply_phi1(sp, nonlinearity(sp, U_start[0]))
    return b


def is_etd1(sp: Spec) -> bool:
    return sp.nl_form == "etd1" and sp.nonlin != "none"


def apply_R(sp: Spec, V: np.ndarray) -> np.ndarray:
    """R_s v: row i is v_i - sum_{j=1..s, i-j>=0} a_j A^j v_{i-j}
    (I - sum_j a_j C_{j-1} (x) A^j with the lower shifts C_{j-1})."""
    a, _ = bdf_float(sp.order)
    out = V.astype(np.result_type(V, np.float64)).copy()
    for i in range(sp.Ns):
        for j in range(1, sp.order + 1):
            if i - j >= 0:
                out[i] -= a[j - 1] * apply_A_power(sp, V[i - j], j)
    return out


def residual(sp: Spec, V: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = f_s + beta dt N(v) - R_s v (Eq. (3.2); the lagged nonlinear term of
    Eq. (7.4) enters with the current iterate).  ETD1: row i >= 1 carries
    dt phi_1(dt L_h) N(v_{i-1}) instead (the previous slice, explicit)."""
    if is_etd1(sp):
        r = b - apply_R(sp, V)
        for i in range(1, sp.Ns):
            r[i] += apply_phi1(sp, nonlinearity(sp, V[i - 1]))
        return r
    _, beta = bdf_float(sp.order)
    return b + beta * sp.dt * nonlinearity(sp, V) - apply_R(sp, V)


def time_eigenvalues(sp: Spec) -> np.ndarray:
    """lambda_{0,n} = alpha^(1/Ns) e^{2 pi i (n-1)/Ns}, n = 1..Ns (Sec. 2)."""
    Ns = sp.Ns
    return sp.alpha ** (1.0 / Ns) * np.exp(2j * np.pi * np.arange(Ns) / Ns)


def gamma_alpha(sp: Spec) -> np.ndarray:
    """Diagonal of Gamma_alpha = diag(1, alpha^(1/Ns), ..., alpha^((Ns-1)/Ns))."""
    return sp.alpha ** (np.arange(sp.Ns) / sp.Ns)


def nonlinearity_derivative(sp: Spec, u: np.ndarray) -> np.ndarray:
    """N'(u): zero for linear problems, 1 - 3 u^2 for Allen-Cahn."""
    if sp.nonlin == "none":
        return np.zeros_like(u)
    if sp.nonlin == "allen_cahn":
        return 1.0 - 3.0 * u**2
    raise ValueError(sp.nonlin)


def jacobian_shift(sp: Spec, u0: np.ndarray) -> float:
    """beta_s dt nbar, nbar the spatial mean of N'(u_0): the inexact Jacobian
    that Sec. 6 proposes after Eq. (6.5), I_t (x) diag(N'(u_0)) (the Jacobian at
    the initial value), averaged over space so that Step (b) stays diagonal in
    L_h's eigenbasis."""
    _, beta = bdf_float(sp.order)
    return beta * sp.dt * float(np.mean(nonlinearity_derivative(sp, u0)))


def precond_apply(sp: Spec, r: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """s = P_alpha^{-1} r by the three steps of Eq. (3.3) / Eq. (4.5).

    Step (a): S_a = (F (x) I)(Gamma_alpha (x) I) r, F the unitary DFT with
              omega = e^{+2 pi i/Ns} (F x = sqrt(Ns) * numpy.ifft(x));
    Step (b): S_b,n = (I - sum_j a_j lambda_n^j A^j)^{-1} S_a,n per slice
              (lambda_{j-1,n} = lambda_{0,n}^j, Sec. 4 after Eq. (4.4)); the spatial solve
              is diagonal in L_h's eigenbasis;
    Step (c): s = (Gamma_alpha^{-1} (x) I)(F^* (x) I) S_b.
    shift != 0 solves with P_alpha - shift I instead (Step (b) of the inexact
    Newton variant, Eq. (6.5), with a scalar Jacobian): per slice
    ((1 - shift) I - sum_j a_j lambda_n^j A^j)^{-1}."""
    Ns = sp.Ns
    a, _ = bdf_float(sp.order)
    gam = gamma_alpha(sp).reshape((Ns,) + (1,) * sp.ndim)
    lam = time_eigenvalues(sp)
    mu = spatial_eigenvalues(sp)
    # Step (a)
    Sa = np.sqrt(Ns) * np.fft.ifft(gam * r, axis=0)
    # Step (b)
    Sb = np.empty_like(Sa)
    for n in range(Ns):
        d = np.full(sp.n, 1.0 - shift, dtype=complex)
        for j in range(1, sp.order + 1):
            d -= a[j - 1] * lam[n] ** j * np.exp(j * sp.dt * mu)
        Sb[n] = from_eigen(sp, to_eigen(sp, Sa[n]) / d)
    # Step (c)
    s = np.fft.fft(Sb, axis=0) / np.sqrt(Ns) / gam
    return s if sp.complex_state else s.real


# ---------------------------------------------------------------------------
# Solvers.
# ---------------------------------------------------------------------------
@dataclass
class SolveResult:
    U: np.ndarray                 # (Nt+1, *n): u_0 .. u_Nt
    iterations: int
    history: List[float]          # relative update / residual norms per iteration
    iterates: Optional[List[np.ndarray]] = None


def assemble(sp: Spec, U_start: np.ndarray, V: np.ndarray) -> np.ndarray:
    U = np.zeros((sp.Nt + 1,) + sp.n, dtype=state_dtype(sp))
    U[: sp.order] = U_start
    U[sp.order:] = V
    return U


def linear_guess(sp: Spec, U_start: np.ndarray) -> np.ndarray:
    """The unknown slices u_s..u_Nt propagated from the last start-up value
    without N and f: u_n = A^{n-s+1} u_{s-1}, A = exp(dt L_h) (Eq. (2.2)).
    This is what the scheme itself produces when N = 0 and f = 0, since the
    BDF coefficients sum to one (Eq. (4.1), Sec. 5): sum_j a_j A^j A^{n-j} u =
    A^n u.  The paper runs the iteration from several initial guesses (Sec. 7)
    without fixing one; this one is the default initial iterate here."""
    u_last = U_start[sp.order - 1]
    return np.stack([apply_A_power(sp, u_last, k + 1) for k in range(sp.Ns)])


def richardson(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None,
               max_iter: int = 50, tol: float = 0.0, keep_iterates: bool = False,
               V0: Optional[np.ndarray] = None,
               U_start: Optional[np.ndarray] = None, jacobian: str = "lagged",
               init: str = "zero") -> SolveResult:
    """Preconditioned fixed-point iteration v^{k+1} = v^k + P_alpha^{-1}(f_s +
    beta dt N(v^k) - R_s v^k) (Eqs. (3.2), (4.4), (7.3)-(7.4)) from v^0 = V0,
    else from zero (init="zero") or from `linear_guess` (init="linear").
    Stops when max_n ||s_n|| <= tol * max_n ||v_n|| or after max_iter
    iterations.  jacobian="mean_u0" preconditions with P_alpha - beta dt nbar I
    (see `jacobian_shift`): the same fixed point, reached by inexact Newton
    steps."""
    shift = jacobian_shift(sp, u0) if jacobian == "mean_u0" else 0.0
    U_start = startup_values(sp, u0, f, U_start)
    b = rhs_known(sp, U_start, f)
    if V0 is not None:
        V = V0.copy()
    elif init == "linear":
        V = linear_guess(sp, U_start)
    elif init == "zero":
        V = np.zeros((sp.Ns,) + sp.n, dtype=state_dtype(sp))
    else:
        raise ValueError(f"unknown initial guess {init!r}")
    hist, its = [], []
    k = 0
    for k in range(1, max_iter + 1):
        s = precond_apply(sp, residual(sp, V, b), shift)
        V = V + s
        sn = np.sqrt((np.abs(s.reshape(sp.Ns, -1)) ** 2).sum(1)).max()
        vn = np.sqrt((np.abs(V.reshape(sp.Ns, -1)) ** 2).sum(1)).max()
        hist.append(sn / vn if vn > 0 else 0.0)
        if keep_iterates:
            its.append(V.copy())
        if hist[-1] <= tol:
            break
    return SolveResult(assemble(sp, U_start, V), k, hist, its if keep_iterates else None)


def gmres(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None, tol: float = 1e-10,
          restart: int = 20, max_iter: int = 200,
          U_start: Optional[np.ndarray] = None) -> SolveResult:
    """Left-preconditioned restarted GMRES(m) with modified Gram-Schmidt on
    P_alpha^{-1} R_s v = P_alpha^{-1} f_s (Sec. 3.2, Theorem 3.3), v^0 = 0.
    Stops when ||P^{-1}(f_s - R_s v)|| <= tol * ||P^{-1} f_s||.
    history[k] is that relative preconditioned residual after k iterations.

    A complex state runs complex GMRES: the Hermitian inner product
    <v, w> = sum conj(v) w, complex Hessenberg entries and complex Givens
    rotations G = [[conj(c), s], [-s, c]] with |c|^2 + s^2 = 1 and s real
    (the subdiagonal entry is a norm); on real data every step reduces to
    the real algorithm."""
    if sp.nonlin != "none":
        raise ValueError("GMRES is for linear problems")
    U_start = startup_values(sp, u0, f, U_start)
    b = rhs_known(sp, U_start, f)
    shape = (sp.Ns,) + sp.n
    dt_ = state_dtype(sp)

    def op(x):
        return precond_apply(sp, apply_R(sp, x.reshape(shape))).ravel()

    c = precond_apply(sp, b).ravel()
    cn = np.linalg.norm(c)
    x = np.zeros_like(c)
    hist = [1.0]
    total = 0
    if cn == 0:
        return SolveResult(assemble(sp, U_start, x.reshape(shape)), 0, hist)
    while total < max_iter:
        r = c - op(x)
        beta = np.linalg.norm(r)
        if beta <= tol * cn:
            break
        m = restart
        Vb = np.zeros((m + 1, c.size), dtype=dt_)
        H = np.zeros((m + 1, m), dtype=dt_)
        cs, sn = np.zeros(m, dtype=dt_), np.zeros(m)
        g = np.zeros(m + 1, dtype=dt_)
        g[0] = beta
        Vb[0] = r / beta
        j_done = 0
        for j in range(m):
            w = op(Vb[j])
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                Vb[j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous Givens rotations
                t = np.conj(cs[i]) * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(abs(H[j, j]), abs(H[j + 1, j]))
            cs[j], sn[j] = H[j, j] / den, abs(H[j + 1, j]) / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            total += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / cn)
            if abs(g[j + 1]) <= tol * cn or total >= max_iter:
                break
        y = scipy.linalg.solve_triangular(H[:j_done, :j_done], g[:j_done])
        x = x + Vb[:j_done].T @ y
        if hist[-1] <= tol:
            break
    return SolveResult(assemble(sp, U_start, x.reshape(shape)), total, hist)


def bicgstab_solve(matvec, b: np.ndarray, tol: float, max_iter: int):
    """BiCGStab (van der Vorst, 1992) for matvec(x) = b from x = 0: the BiCG
    direction step followed by a one-dimensional minimal residual step each
    iteration, with the Hermitian products <u, v> = sum conj(u) v (plain dot
    products on real data).  Stops when ||r_k|| <= tol ||b||; on a breakdown
    (rho exactly zero) it restarts the shadow residual rhat = r.
    Returns (x, history of ||r_k|| / ||b||)."""
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = [1.0]
    if bn == 0:
        return x, hist
    r = b.copy()
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(max_iter):
        rho_new = np.vdot(rhat, r)
        if rho_new == 0.0:                     # breakdown: restart the shadow residual
            rhat = r.copy()
            rho, alpha, omega = 1.0, 1.0, 1.0
            v[:] = 0.0
            p[:] = 0.0
            rho_new = np.vdot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho_new / np.vdot(rhat, v)
        s = r - alpha * v
        t = matvec(s)
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        hist.append(float(np.linalg.norm(r)) / bn)
        if hist[-1] <= tol:
            break
    return x, hist


def bicgstab(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None, tol: float = 1e-10,
             max_iter: int = 200, U_start: Optional[np.ndarray] = None) -> SolveResult:
    """Left-preconditioned BiCGStab on P_alpha^{-1} R_s v = P_alpha^{-1} f_s
    (the Krylov alternative to GMRES timed in Sec. 7, Table 2), v^0 = 0,
    with the same stopping rule as `gmres`."""
    if sp.nonlin != "none":
        raise ValueError("BiCGStab is for linear problems")
    U_start = startup_values(sp, u0, f, U_start)
    b = rhs_known(sp, U_start, f)
    shape = (sp.Ns,) + sp.n

    def op(x):
        return precond_apply(sp, apply_R(sp, x.reshape(shape))).ravel()

    x, hist = bicgstab_solve(op, precond_apply(sp, b).ravel(), tol, max_iter)
    return SolveResult(assemble(sp, U_start, x.reshape(shape)), len(hist) - 1, hist)


# ---------------------------------------------------------------------------
# Error metric: L^inf(0,T; L^2) relative error (Sec. 7).
# ---------------------------------------------------------------------------
def rel_error(U: np.ndarray, Uref: np.ndarray) -> float:
    """max_n ||u_n - u_n^ref||_2 / max_n ||u_n^ref||_2 over the given slices."""
    d = np.abs(U - Uref).reshape(U.shape[0], -1)
    r = np.abs(Uref).reshape(Uref.shape[0], -1)
    return float(np.sqrt((d**2).sum(1)).max() / np.sqrt((r**2).sum(1)).max())


# ---------------------------------------------------------------------------
# Dense brute force for tiny sizes (independent of the eigen-symbol path).
# ---------------------------------------------------------------------------
def dense_laplacian_1d(bc: str, n: int, L: float) -> np.ndarray:
    """Periodic: the spectral second-derivative matrix of the periodic sinc
    interpolant (even n): -pi^2/(3h^2) - 1/6 on the diagonal and
    -(-1)^j / (2 sin^2(j h/2)) off it, for the grid spacing h = 2 pi/n, scaled
    to length L.  Dirichlet: tridiag(1, -2, 1)/h^2 with h = L/(n+1).  Neumann:
    the same on n cell centres, h = L/n, with the mirrored ghost values
    u_0 = u_1 and u_{n+1} = u_n folding the outer couplings onto the first
    and last diagonal entries (-1/h^2)."""
    if bc == PERIODIC:
        if n % 2:
            raise ValueError("even n only")
        h = 2.0 * np.pi / n
        col = np.empty(n)
        col[0] = -np.pi**2 / (3.0 * h**2) - 1.0 / 6.0
        j = np.arange(1, n)
        col[1:] = -((-1.0) ** j) / (2.0 * np.sin(j * h / 2.0) ** 2)
        return scipy.linalg.toeplitz(col) * (2.0 * np.pi / L) ** 2
    h = L / n if bc == NEUMANN else L / (n + 1)
    T = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    if bc == NEUMANN:
        T[0, 0] += 1.0
        T[-1, -1] += 1.0
    return T / h**2


def dense_derivative_1d(n: int, L: float) -> np.ndarray:
    """Periodic spectral first-derivative matrix of the sinc interpolant (even
    n): D[j, k] = (-1)^(j-k) cot((j - k) h/2)/2 off the diagonal, 0 on it
    (h = 2 pi/n), scaled to length L; its eigenvalues are i*2 pi k/L for
    |k| < n/2 and 0 at n/2."""
    if n % 2:
        raise ValueError("even n only")
    h = 2.0 * np.pi / n
    col = np.zeros(n)
    j = np.arange(1, n)
    col[1:] = 0.5 * ((-1.0) ** j) / np.tan(j * h / 2.0)   # D[j, 0]
    row = col[(-np.arange(n)) % n]                         # D[0, k] = D[n - k, 0]
    return scipy.linalg.toeplitz(col, row) * (2.0 * np.pi / L)


def dense_Lh(sp: Spec) -> np.ndarray:
    """L_h = a Delta_h - b.grad_h - c I as an explicit matrix (row-major grid ordering)."""
    mats = [dense_laplacian_1d(sp.bc, n, L) for n, L in zip(sp.n, sp.length)]
    M = int(np.prod(sp.n))

    def embed(D, d):
        term = np.ones((1, 1))
        for e in range(sp.ndim):
            term = np.kron(term, D if e == d else np.eye(sp.n[e]))
        return term

    lap = np.zeros((M, M))
    for d, D in enumerate(mats):
        lap += embed(D, d)
    out = sp.a * lap - sp.c * np.eye(M)
    if has_advection(sp):
        for d, (n, L) in enumerate(zip(sp.n, sp.length)):
            if d < len(sp.b) and sp.b[d] != 0.0:
                out -= sp.b[d] * embed(dense_derivative_1d(n, L), d)
    return out


def dense_A(sp: Spec) -> np.ndarray:
    """A = exp(dt L_h) by scipy's scaling-and-squaring expm."""
    return scipy.linalg.expm(sp.dt * dense_Lh(sp))


def dense_phi1(sp: Spec) -> np.ndarray:
    """dt phi_1(dt L_h) from one expm of the augmented matrix
    [[dt L_h, I], [0, 0]], whose top-right block is sum_k (dt L_h)^k/(k+1)!
    = phi_1(dt L_h): independent of the eigen-symbol path."""
    Z = sp.dt * dense_Lh(sp)
    M = Z.shape[0]
    aug = np.zeros((2 * M, 2 * M))
    aug[:M, :M] = Z
    aug[:M, M:] = np.eye(M)
    return sp.dt * scipy.linalg.expm(aug)[:M, M:]


def shift_matrix(N: int, j: int, alpha: float = 0.0) -> np.ndarray:
    """C_j (alpha = 0) or C_j^alpha: ones where row - col = j+1, and alpha on
    the wrap-around entries row - col = j+1-N (top-right corner).
    C_0^alpha is Eq. (2.4); C_1^alpha has alpha at (1, N-1) and (2, N)
    (Sec. 4 after Eq. (4.4), 1-based); C_j^alpha for j >= 2 is read as
    (C_0^alpha)^(j+1) (the entry lists printed in Sec. 5 are garbled)."""
    C = np.zeros((N, N))
    for r in range(N):
        cidx = r - (j + 1)
        if cidx >= 0:
            C[r, cidx] = 1.0
        else:
            C[r, cidx + N] = alpha
    return C


def dense_R(sp: Spec, alpha: float = 0.0) -> np.ndarray:
    """R_s (alpha = 0) or R_s^alpha = I - sum_j a_j C_{j-1}^alpha (x) A^j."""
    a, _ = bdf_float(sp.order)
    A = dense_A(sp)
    M = A.shape[0]
    Ns = sp.Ns
    R = np.eye(Ns * M, dtype=A.dtype)
    Aj = np.eye(M, dtype=A.dtype)
    for j in range(1, sp.order + 1):
        Aj = Aj @ A
        R -= a[j - 1] * np.kron(shift_matrix(Ns, j - 1, alpha), Aj)
    return R


def dense_rhs(sp: Spec, U_start: np.ndarray, f: Optional[np.ndarray]) -> np.ndarray:
    """f_s assembled with the dense A (the printed f_2..f_6 plus the source)."""
    a, beta = bdf_float(sp.order)
    A = dense_A(sp)
    s = sp.order
    M = A.shape[0]
    b = np.zeros((sp.Ns, M), dtype=np.result_type(A, U_start, state_dtype(sp)))
    for i in range(sp.Ns):
        n = s + i
        if f is not None:
            b[i] += beta * sp.dt * f[n - 1].ravel()
        for j in range(1, s + 1):
            if n - j < s:
                b[i] += a[j - 1] * (np.linalg.matrix_power(A, j) @ U_start[n - j].ravel())
    return b.ravel()


def dense_solve(sp: Spec, u0: np.ndarray, f: Optional[np.ndarray] = None) -> np.ndarray:
    """u_0..u_Nt from the dense all-at-once system.  Linear: one LU solve of
    R_s v = f_s.  Allen-Cahn: Newton on R_s v - beta dt N(v) = f_s with the
    dense Jacobian.  The startup ramp is stepped with the dense A too."""
    a, _ = bdf_float(sp.order)
    A = dense_A(sp)
    M = A.shape[0]
    if is_etd1(sp):
        return _dense_solve_etd1(sp, u0, f, A)
    # dense startup ramp u_1..u_{s-1}
    Us = [u0.ravel().copy()]
    for n in range(1, sp.order):
        an, bn = bdf_float(n)
        w = sum(an[j - 1] * (np.linalg.matrix_power(A, j) @ Us[n - j]) for j in range(1, n + 1))
        if f is not None:
            w = w + bn * sp.dt * f[n - 1].ravel()
        Us.append(_dense_pointwise(sp, w, bn * sp.dt))
    U_start = np.array(Us).reshape((sp.order,) + sp.n)
    b = dense_rhs(sp, U_start, f)
    R = dense_R(sp)
    _, beta = bdf_float(sp.order)
    if sp.nonlin == "none":
        v = scipy.linalg.lu_solve(scipy.linalg.lu_factor(R), b)
    else:
        v = np.linalg.solve(R, b)
        for _ in range(50):
            F = R @ v - beta * sp.dt * (v - v**3) - b
            J = R - beta * sp.dt * np.diag(1.0 - 3.0 * v**2)
            dv = np.linalg.solve(J, F)
            v = v - dv
            if np.max(np.abs(dv)) < 1e-15:
                break
    return assemble(sp, U_start, v.reshape((sp.Ns,) + sp.n))


def _dense_solve_etd1(sp: Spec, u0: np.ndarray, f, A: np.ndarray) -> np.ndarray:
    """ETD1 as one dense all-at-once system: R_1 v - (C_0 (x) Phi) N(v) = b
    with b_0 = A u_0 + Phi N(u_0), Phi = dt phi_1(dt L_h) from dense_phi1,
    solved by Newton with the dense Jacobian from v = 0."""
    _check_etd1(sp, f)
    Phi = dense_phi1(sp)
    M = A.shape[0]
    Ns = sp.Ns
    R = dense_R(sp)
    S = np.kron(shift_matrix(Ns, 0), Phi)
    u0v = u0.ravel()
    b = np.zeros(Ns * M)
    b[:M] = A @ u0v + Phi @ (u0v - u0v**3)
    v = np.zeros(Ns * M)
    for _ in range(60):
        F = R @ v - S @ (v - v**3) - b
        J = R - S @ np.diag(1.0 - 3.0 * v**2)
        dv = np.linalg.solve(J, F)
        v = v - dv
        if np.max(np.abs(dv)) < 1e-15:
            break
    return assemble(sp, u0[None], v.reshape((Ns,) + sp.n))


def _dense_pointwise(sp: Spec, w: np.ndarray, bdt: float) -> np.ndarray:
    if sp.nonlin == "none":
        return w
    u = w.copy()
    for _ in range(60):
        du = (u - bdt * (u - u**3) - w) / (1.0 - bdt + 3.0 * bdt * u**2)
        u = u - du
        if np.max(np.abs(du)) < 1e-16:
            break
    return u


def dense_precond_apply(sp: Spec, r: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """(P_alpha - shift I)^{-1} r by an LU solve with the explicit dense R_s^alpha."""
    P = dense_R(sp, sp.alpha)
    return np.linalg.solve(P - shift * np.eye(P.shape[0]), r.ravel()).reshape(r.shape)


def dense_iteration_matrix(sp: Spec) -> np.ndarray:
    """I - (R_s^alpha)^{-1} R_s, the Richardson iteration matrix (Eq. (3.4))."""
    R = dense_R(sp)
    Ra = dense_R(sp, sp.alpha)
    return np.eye(R.shape[0]) - np.linalg.solve(Ra, R)
