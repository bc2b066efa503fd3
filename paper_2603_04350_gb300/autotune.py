"""Per-shape choice among the library's interchangeable kernel variants.

libexpd carries more than one kernel for several steps of the hot path, each
computing the same result (the GPU tests check each pair):

  fft   periodic spatial FFTs: four-step register kernels (default) or the
        shared-memory radix-4 kernels (EXPD_KF_FFT_RADIX4)
  time  the time-direction kernel for windows of 16, 32 or 64 unknown slices
        on the mixed path: register kernel (default) or the shared-memory
        kernel (EXPD_KF_TIME_SMEM)
  dst   dense sine transforms on the mixed path (2D Dirichlet, sizes multiples
        of 128 up to 1024): split-bf16 digit products on the tensor cores in
        128 x 128 output tiles (default) or 128 x 64 tiles (EXPD_KF_DST_N64,
        twice the tiles for grids too small to fill the SMs), or float64
        products (EXPD_KF_DST_FP64)

Which is faster depends on the grid, the window and the precision.  A Tuner
times every applicable combination on the device (whole solves, CUDA events,
the median of a few after warm-up), keeps the fastest per problem shape, and
creates plans with it.  The choice travels to the library as the scheme's
kernel_flags bits, per plan, so tuned and untuned plans can be created from
any thread at the same time.  Choices persist as JSON (save / load).
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import statistics
import threading
from typing import Callable, Dict, List, Optional, Tuple

from . import expd
from . import inputs as I

ALL_FLAGS = expd.KF_TIME_SMEM | expd.KF_FFT_RADIX4 | expd.KF_DST_FP64 | expd.KF_DST_N64
KNOBS: Dict[str, Tuple[Tuple[str, int], ...]] = {
    "fft": (("four_step", 0), ("radix4", expd.KF_FFT_RADIX4)),
    "time": (("register", 0), ("smem", expd.KF_TIME_SMEM)),
    "dst": (("tensor", 0), ("tensor_n64", expd.KF_DST_N64), ("float64", expd.KF_DST_FP64)),
}


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


def candidates(p: I.Problem, precision: int) -> List[Tuple[Dict[str, str], int]]:
    """Every combination of the applicable variants: (names, kernel_flags)."""
    names = knobs_for(p, precision)
    out = []
    for combo in itertools.product(*(KNOBS[k] for k in names)):
        choice = {k: c[0] for k, c in zip(names, combo)}
        flags = 0
        for c in combo:
            flags |= c[1]
        out.append((choice, flags))
    return out


def shape_key(p: I.Problem, precision: int, solver: str) -> str:
    """What the choice depends on: boundary, grid, window, order, nonlinearity, precision, solver."""
    return "|".join(str(v) for v in (p.bc, "x".join(map(str, p.n)), p.Nt, p.order, p.nonlin, precision, solver))


def with_flags(spec: expd.PlanSpec, flags: Optional[int]) -> expd.PlanSpec:
    """The spec with exactly these variant bits (None: the defaults, 0)."""
    return dataclasses.replace(spec, kernel_flags=int(flags or 0))


def plan_create(spec: expd.PlanSpec, flags: Optional[int], stream=None) -> expd.Plan:
    """expd.plan_create with the given kernel variants (None: the defaults)."""
    return expd.plan_create(with_flags(spec, flags), stream)


def measure_solves(p: I.Problem, precision: int, solver: str, flags: int, reps: int = 3,
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
        with plan_create(spec, flags, stream) as plan:
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

    measure(p, precision, solver, flags) -> milliseconds; the default times
    whole solves on the GPU (measure_solves)."""

    def __init__(self, measure: Optional[Callable[..., float]] = None, reps: int = 3, warmup: int = 1):
        self.measure = measure or (lambda p, prec, solver, fl: measure_solves(p, prec, solver, fl, reps, warmup))
        self.table: Dict[str, dict] = {}
        self._lock = threading.Lock()

    def tune(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> dict:
        """Times every candidate for this shape (even if cached) and records the fastest."""
        solver = solver or p.solver
        trials = []
        for choice, flags in candidates(p, precision):
            trials.append({"choice": choice, "flags": flags, "ms": float(self.measure(p, precision, solver, flags))})
        best = min(trials, key=lambda t: t["ms"]) if trials else {"choice": {}, "flags": 0, "ms": None}
        entry = {"choice": best["choice"], "flags": best["flags"], "ms": best["ms"], "trials": trials}
        with self._lock:
            self.table[shape_key(p, precision, solver)] = entry
        return entry

    def lookup(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> Optional[int]:
        """The recorded best kernel_flags for this shape, or None (never measures)."""
        with self._lock:
            e = self.table.get(shape_key(p, precision, solver or p.solver))
        return int(e["flags"]) if e else None

    def best(self, p: I.Problem, precision: int, solver: Optional[str] = None) -> int:
        flags = self.lookup(p, precision, solver)
        return flags if flags is not None else int(self.tune(p, precision, solver)["flags"])

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
            if not isinstance(e, dict) or not isinstance(e.get("flags"), int) or isinstance(e.get("flags"), bool) \
                    or e["flags"] & ~ALL_FLAGS or e["flags"] < 0:
                raise ValueError(f"autotune table entry {k!r} is malformed")
        with self._lock:
            self.table.update(data)
