"""Per-shape choice among the library's interchangeable kernel variants.

libexpd carries more than one kernel for several steps of the hot path, each
computing the same result (the GPU tests check each pair):

  fft   periodic spatial FFTs: four-step register kernels (default) or the
        shared-memory radix-4 kernels (EXPD_FFT_KERNEL=radix4)
  time  the time-direction kernel for windows of 16, 32 or 64 unknown slices
        on the mixed path: register kernel (default) or the shared-memory
        kernel (EXPD_TIME_KERNEL=smem)
  dst   dense sine transforms on the mixed path (2D Dirichlet, sizes multiples
        of 128 up to 1024): split-bf16 digit products on the tensor cores
        (default) or float64 products (EXPD_DST_TC=0)

Which is faster depends on the grid, the window and the precision.  A Tuner
times every applicable combination on the device (whole solves, CUDA events,
the median of a few after warm-up), keeps the fastest per problem shape, and
creates plans with it.  The variant switches are read when a plan is created,
so plan_create() holds a process-wide lock while it sets them; solves run
without it.  Choices persist as JSON (save / load).
"""
from __future__ import annotations

import contextlib
import itertools
import json
import os
import statistics
import threading
from typing import Callable, Dict, List, Optional, Tuple

from . import expd
from . import inputs as I

ENV_NAMES = ("EXPD_FFT_KERNEL", "EXPD_TIME_KERNEL", "EXPD_DST_TC")
KNOBS: Dict[str, Tuple[Tuple[str, Dict[str, str]], ...]] = {
    "fft": (("four_step", {}), ("radix4", {"EXPD_FFT_KERNEL": "radix4"})),
    "time": (("register", {}), ("smem", {"EXPD_TIME_KERNEL": "smem"})),
    "dst": (("tensor", {}), ("float64", {"EXPD_DST_TC": "0"})),
}
_ENV_LOCK = threading.Lock()


def _pow2(n: int) -> bool:
    return n > 0 and (n & (n - 1)) == 0


def knobs_for(p: I.Problem, precision: int) -> List[str]:
    """The switches that select between different kernels for this problem."""
    out = []
    if p.bc == "periodic":
        out.append("fft")
    ns = p.Nt - p.order + 1
    if precision == expd.PREC_MIXED and ns in (16, 32, 64):
        out.append("time")
    if (p.bc == "dirichlet" and precision == expd.PREC_MIXED and len(p.n) == 2
            and all(n % 128 == 0 and n <= 1024 and not _pow2(n + 1) for n in p.n)):
        out.append("dst")
    return out


def candidates(p: I.Problem, precision: int) -> List[Tuple[Dict[str, str], Dict[str, str]]]:
    """Every combination of the applicable variants: (names, environment)."""
    names = knobs_for(p, precision)
    out = []
    for combo in itertools.product(*(KNOBS[k] for k in names)):
        choice = {k: c[0] for k, c in zip(names, combo)}
        env: Dict[str, str] = {}
        for c in combo:
            env.update(c[1])
        out.append((choice, env))
    return out


def shape_key(p: I.Problem, precision: int, solver: str) -> str:
    """What the choice depends on: boundary, grid, window, order, nonlinearity, precision, solver."""
    return "|".join(str(v) for v in (p.bc, "x".join(map(str, p.n)), p.Nt, p.order, p.nonlin, precision, solver))


@contextlib.contextmanager
def variant_env(env: Dict[str, str]):
    """Sets exactly the given switches (clearing the others) under the process-wide lock."""
    with _ENV_LOCK:
        saved = {k: os.environ.get(k) for k in ENV_NAMES}
        try:
            for k in ENV_NAMES:
                os.environ.pop(k, None)
            os.environ.update(env)
            yield
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v


def plan_create(spec: expd.PlanSpec, env: Optional[Dict[str, str]], stream=None) -> expd.Plan:
    """expd.plan_create with the given variant switches (None: the defaults)."""
    with variant_env(env or {}):
        return expd.plan_create(spec, stream)


def measure_solves(p: I.Problem, precision: int, solver: str, env: Dict[str, str], reps: int = 3,
                   warmup: int = 1, device: int = 0) -> float:
    """Median milliseconds of `reps` whole solves (after `warmup`), CUDA events on the solve stream."""
    import torch

    dev = torch.device("cuda", device)
    u0, f = I.make_inputs(p)
    u0d = torch.from_numpy(u0).to(dev)
    fd = torch.from_numpy(f).to(dev) if f is not None else None
    U = torch.empty((p.Nt,) + tuple(p.n), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    spec = expd.spec_from_problem(p, precision=precision, max_iter=200)
    ms = []
    with torch.cuda.stream(stream):
        with plan_create(spec, env, stream) as plan:
            fn = {"fp": plan.solve_fp, "gmres": plan.solve_gmres, "bicgstab": plan.solve_bicgstab}[solver]
            for k in range(warmup + reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn(u0d, fd, U, stream)
                e1.record(stream)
                stream.synchronize()
                if k >= warmup:
                    ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


class Tuner:
    """Fastest variant per problem shape, measured on first request and cached.

    measure(p, precision, solver, env) -> milliseconds; the default times whole
    solves on the GPU (measure_solves)."""

    def __init__(self, measure: Optional[Callable[..., float]] = None, reps: int = 3, warmup: int = 1):
        self.measure = measure or (lambda p, prec, solver, env: measure_solves(p, prec, solver, env, reps, warmup))
        self.table: Dict[str, dict] = {}
        self._lock = threading.Lock()

    def tune(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> dict:
        """Times every candidate for this shape (even if cached) and records the fastest."""
        solver = solver or p.solver
        trials = []
        for choice, env in candidates(p, precision):
            trials.append({"choice": choice, "env": env, "ms": float(self.measure(p, precision, solver, env))})
        best = min(trials, key=lambda t: t["ms"]) if trials else {"choice": {}, "env": {}, "ms": None}
        entry = {"choice": best["choice"], "env": best["env"], "ms": best["ms"], "trials": trials}
        with self._lock:
            self.table[shape_key(p, precision, solver)] = entry
        return entry

    def lookup(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> Optional[Dict[str, str]]:
        """The recorded best switches for this shape, or None (never measures)."""
        with self._lock:
            e = self.table.get(shape_key(p, precision, solver or p.solver))
        return dict(e["env"]) if e else None

    def best(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> Dict[str, str]:
        env = self.lookup(p, precision, solver)
        return env if env is not None else dict(self.tune(p, precision, solver)["env"])

    def plan_create(self, p: I.Problem, spec: expd.PlanSpec, stream=None, solver: Optional[str] = None) -> expd.Plan:
        """A plan for problem p with its recorded best variants (the defaults when none is recorded)."""
        return plan_create(spec, self.lookup(p, spec.precision, solver), stream)

    def save(self, path: str) -> None:
        with self._lock:
            data = dict(self.table)
        with open(path, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)

    def load(self, path: str) -> None:
        with open(path) as fh:
            data = json.load(fh)
        for k, e in data.items():
            if not isinstance(e, dict) or not isinstance(e.get("env"), dict) or \
                    any(n not in ENV_NAMES for n in e["env"]):
                raise ValueError(f"autotune table entry {k!r} is malformed")
        with self._lock:
            self.table.update(data)
