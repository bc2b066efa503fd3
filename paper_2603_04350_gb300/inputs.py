"""Seeded synthetic workloads for Exp-ParaDiag.

This module holds problem parameters and seeded input generators only; it
contains none of the method's arithmetic (no exponential, no time stepping, no
preconditioner).  It is the one module that both the CUDA path's callers and
the CPU oracle's tests draw their inputs from.

The paper (Sec. 6) runs synthetic PDE problems and uses no dataset, so every
input here is generated from a seed.  The five workloads follow the problem
classes of the paper: periodic heat (exact-solution check, Sec. 6.1),
periodic Allen-Cahn u_t = eps^2 Lap u + u - u^3 (Sec. 6.2, lagged form of
Eq. (6.2)), and the 2D Dirichlet heat equation of Table 2 with a smooth source.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

PERIODIC = "periodic"
DIRICHLET = "dirichlet"
NEUMANN = "neumann"
NL_NONE = "none"
NL_ALLEN_CAHN = "allen_cahn"


@dataclass(frozen=True)
class Problem:
    """Parameters of one all-at-once solve.

    n       grid points per dimension (periodic), interior points (Dirichlet)
            or cells (Neumann)
    length  domain length per dimension; periodic grid x_j = j*L/n,
            Dirichlet grid x_j = j*L/(n+1), j = 1..n, Neumann cell centres
            x_j = (j - 1/2) L/n
    a, c    L = a*Lap - c  (Sec. 1, Eq. (1.2)); b adds advection -b.grad; a and c
            may be complex (the Schrodinger equation of Sec. 7: a = i, c = 2i
            or 200i), which needs complex_state
    nonlin  N(u): "none" or "allen_cahn" (N(u) = u - u^3)
    dt, Nt  time step and number of steps; the window is T = Nt*dt
    alpha   the alpha-circulant parameter (Sec. 2)
    order   exponential BDF order s in 1..6 (Secs. 3-5)
    """

    name: str
    bc: str
    n: Tuple[int, ...]
    length: Tuple[float, ...]
    a: float
    c: float
    nonlin: str
    dt: float
    Nt: int
    alpha: float
    order: int
    tol: float = 1e-8
    solver: str = "fp"          # "fp" (Richardson) or "gmres"
    seed: int = 0
    forcing: bool = False
    u0_kind: str = "uniform"
    u0_range: Tuple[float, float] = (-0.9, 0.9)
    u0_lowpass: Optional[int] = None
    b: Tuple[float, ...] = ()   # advection velocity per axis (periodic): L = a*Lap - b.grad - c
    nl_form: str = "if"         # nonlinear term: "if" (integrating factor) or "etd1" (order 1, no source)
    complex_state: bool = False  # u0, f and the solution are complex128

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def M(self) -> int:
        return int(np.prod(self.n))

    @property
    def Ns(self) -> int:
        """Number of unknown slices u_s..u_Nt of the all-at-once system."""
        return self.Nt - self.order + 1

    @property
    def unknowns(self) -> int:
        return self.Ns * self.M

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes are the full ones; tests shrink them with .with_().
# ---------------------------------------------------------------------------
HEAT1D = Problem(
    name="heat1d_periodic_n128_nt32_s1", bc=PERIODIC, n=(128,), length=(2 * math.pi,),
    a=1.0, c=0.0, nonlin=NL_NONE, dt=1.0 / 32, Nt=32, alpha=1e-2, order=1, tol=1e-8,
    solver="fp", seed=1, u0_kind="fourier16",
)
ALLEN_CAHN_256 = Problem(
    name="allen_cahn_periodic_256x256_nt64_s1", bc=PERIODIC, n=(256, 256), length=(1.0, 1.0),
    a=0.05 ** 2, c=0.0, nonlin=NL_ALLEN_CAHN, dt=1e-3, Nt=64, alpha=1e-3, order=1, tol=1e-8,
    solver="fp", seed=2, u0_kind="uniform", u0_range=(-0.9, 0.9),
)
HEAT_DIRICHLET_1024 = Problem(
    name="heat_dirichlet_1024x1024_nt128_s2", bc=DIRICHLET, n=(1024, 1024), length=(1.0, 1.0),
    a=1.0, c=0.0, nonlin=NL_NONE, dt=0.1 / 128, Nt=128, alpha=1e-3, order=2, tol=1e-9,
    solver="gmres", seed=3, forcing=True, u0_kind="gaussian",
)
ALLEN_CAHN_512_S6 = Problem(
    name="allen_cahn_periodic_512x512_nt256_s6", bc=PERIODIC, n=(512, 512), length=(1.0, 1.0),
    a=0.02 ** 2, c=0.0, nonlin=NL_ALLEN_CAHN, dt=1e-3, Nt=256, alpha=1e-3, order=6, tol=1e-8,
    solver="fp", seed=4, u0_kind="uniform", u0_range=(-1.0, 1.0), u0_lowpass=32,
)
# The Schrodinger equation u_t = i Lap u - c u of Sec. 7 (a = i), homogeneous
# Dirichlet conditions on the unit interval / square, alpha = alpha_opt =
# 1/5120 (the table of optimised alpha in Sec. 7), GMRES.  1D: h = 1/128
# (127 interior points), dt = 0.01, c = 2i, u_0 = sin(pi x), first order,
# T = 2.  2D: h = 1/40 (39^2 interior points), dt = 0.05, c = 200i, BDF2,
# the Gaussian wave packet u_0 = exp(-|x - 1/2|^2/(2 mu^2)) exp(-5i (x - 1/2)),
# mu = 0.05, T = 4.  The paper stops at an error of 1e-10 (Sec. 7).
ALPHA_OPT = 1.0 / 5120.0
SCHRODINGER_1D = Problem(
    name="schrodinger_dirichlet_127_nt200_s1", bc=DIRICHLET, n=(127,), length=(1.0,),
    a=1j, c=2j, nonlin=NL_NONE, dt=0.01, Nt=200, alpha=ALPHA_OPT, order=1, tol=1e-10,
    solver="gmres", seed=6, u0_kind="sine_mode", complex_state=True,
)
SCHRODINGER_2D = Problem(
    name="schrodinger_dirichlet_39x39_nt80_s2", bc=DIRICHLET, n=(39, 39), length=(1.0, 1.0),
    a=1j, c=200j, nonlin=NL_NONE, dt=0.05, Nt=80, alpha=ALPHA_OPT, order=2, tol=1e-10,
    solver="gmres", seed=7, u0_kind="wave_packet", complex_state=True,
)
WORKLOADS = {p.name: p for p in (HEAT1D, ALLEN_CAHN_256, HEAT_DIRICHLET_1024, ALLEN_CAHN_512_S6,
                                 SCHRODINGER_1D, SCHRODINGER_2D)}


def grid_coords(p: Problem):
    """Per-dimension grid coordinates (1D arrays)."""
    out = []
    for n, L in zip(p.n, p.length):
        if p.bc == PERIODIC:
            out.append(np.arange(n) * (L / n))
        elif p.bc == NEUMANN:
            out.append((np.arange(n) + 0.5) * (L / n))       # cell centres
        else:
            out.append(np.arange(1, n + 1) * (L / (n + 1)))
    return out


def make_u0(p: Problem) -> np.ndarray:
    """Seeded initial state of shape p.n (float64; complex128 for complex states)."""
    u = _make_u0(p)
    return u.astype(np.complex128) if p.complex_state else u


def _make_u0(p: Problem) -> np.ndarray:
    rng = np.random.default_rng(p.seed)
    xs = grid_coords(p)
    if p.u0_kind == "fourier16":
        # 16 Fourier modes with N(0,1) coefficients scaled by k^-2, no k=0 mode.
        x = xs[0]
        ak = rng.standard_normal(16)
        bk = rng.standard_normal(16)
        u = np.zeros_like(x)
        for k in range(1, 17):
            u += (ak[k - 1] * np.cos(k * x) + bk[k - 1] * np.sin(k * x)) / k**2
        return u
    if p.u0_kind == "uniform":
        lo, hi = p.u0_range
        u = rng.uniform(lo, hi, size=p.n)
        if p.u0_lowpass is not None:
            u = lowpass(u, p.u0_lowpass)
        return u
    if p.u0_kind == "gaussian":
        grids = np.meshgrid(*xs, indexing="ij")
        r2 = sum((g - 0.5 * L) ** 2 for g, L in zip(grids, p.length))
        return np.exp(-20.0 * r2)
    if p.u0_kind == "sine_mode":
        # single grid sine mode sin(pi*x)*sin(2*pi*y)... (used by tests)
        grids = np.meshgrid(*xs, indexing="ij")
        u = np.ones(p.n)
        for d, g in enumerate(grids):
            u = u * np.sin((d + 1) * math.pi * g / p.length[d])
        return u
    if p.u0_kind == "constant":
        return np.full(p.n, p.u0_range[0])
    if p.u0_kind == "wave_packet":
        # Gaussian of width mu = 0.05 centred in the domain, carrying the
        # phase exp(-5i (x - L_x/2)) along the first axis
        grids = np.meshgrid(*xs, indexing="ij")
        r2 = sum((g - 0.5 * L) ** 2 for g, L in zip(grids, p.length))
        mu = 0.05
        return np.exp(-r2 / (2.0 * mu * mu)) * np.exp(-5j * (grids[0] - 0.5 * p.length[0]))
    if p.u0_kind == "random_complex":
        return rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    raise ValueError(p.u0_kind)


def lowpass(u: np.ndarray, kmax: int) -> np.ndarray:
    """Keep Fourier modes with |k_d| <= kmax in every dimension; zero the
    Nyquist modes so the result stays real and Hermitian-consistent."""
    uh = np.fft.fftn(u)
    keep = np.ones(u.shape, dtype=bool)
    for d, n in enumerate(u.shape):
        k = np.fft.fftfreq(n, 1.0 / n)
        kd = np.abs(k) <= kmax
        if n % 2 == 0:
            kd &= (k != -n // 2)
        shape = [1] * u.ndim
        shape[d] = n
        keep &= kd.reshape(shape)
    return np.fft.ifftn(uh * keep).real


def forcing_modes(p: Problem):
    """(c_i, p_i, q_i) of the source f = e^{-t} sum_i c_i sin(p_i pi x) sin(q_i pi y)."""
    rng = np.random.default_rng(p.seed)
    c = rng.standard_normal(4)
    pq = rng.integers(1, 9, size=(4, p.ndim))
    return c, pq


def make_forcing(p: Problem) -> Optional[np.ndarray]:
    """Source f(t_n, x) for n = 1..Nt, shape (Nt, *p.n), or None."""
    if not p.forcing:
        return None
    c, pq = forcing_modes(p)
    xs = grid_coords(p)
    grids = np.meshgrid(*xs, indexing="ij")
    g = np.zeros(p.n)
    for i in range(len(c)):
        term = np.full(p.n, c[i])
        for d, gd in enumerate(grids):
            term = term * np.sin(pq[i, d] * math.pi * gd / p.length[d])
        g += term
    t = np.arange(1, p.Nt + 1) * p.dt
    f = np.exp(-t).reshape((-1,) + (1,) * p.ndim) * g[None]
    return f.astype(np.complex128) if p.complex_state else f


def make_inputs(p: Problem):
    """(u0, f) for a problem: u0 of shape p.n, f of shape (Nt, *p.n) or None."""
    return make_u0(p), make_forcing(p)


# ---------------------------------------------------------------------------
# The served mix: seeded Poisson arrivals of heterogeneous requests.
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    problem: Problem


def served_mix(count: int = 2000, seed: int = 5, rate_per_s: float = 100.0,
               grids=(64, 128, 256, 512, 1024), nts=(16, 32, 64, 128, 256), orders=(1, 2, 6)):
    """Requests with Poisson arrivals; kind, grid, Nt and order drawn uniformly.

    Heat requests are Dirichlet: the 1024^2 Dirichlet workload's parameters
    (GMRES, tol 1e-9, the smooth source) with the drawn sizes, a grid g^2 being
    g x g interior points as in that workload; Allen-Cahn requests are
    periodic (the 256^2 workload's parameters with the drawn sizes, fixed
    point, tol 1e-8)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    reqs = []
    for i in range(count):
        kind = int(rng.integers(0, 2))
        g = int(rng.choice(grids))
        nt = int(rng.choice(nts))
        s = int(rng.choice(orders))
        rseed = int(rng.integers(0, 2**31 - 1))
        if kind == 0:
            base = HEAT_DIRICHLET_1024
            prob = base.with_(name=f"req{i}_heat_{g}_{nt}_{s}", n=(g, g), Nt=nt, dt=0.1 / nt,
                              order=s, seed=rseed)
        else:
            base = ALLEN_CAHN_256
            prob = base.with_(name=f"req{i}_ac_{g}_{nt}_{s}", n=(g, g), Nt=nt, order=s,
                              seed=rseed)
        reqs.append(Request(i, float(t[i]), prob))
    return reqs
