"""Served mix: continuous batching of independent solves on one GPU.

Requests differ in kind (periodic Allen-Cahn or Dirichlet heat), grid, Nt and
scheme order, and arrive over time.  The engine keeps the GPU busy with
several of them at once:

* a pool of worker threads, each with its own CUDA stream (the C ABI releases
  the GIL, so solves on different streams overlap on the device);
* admission against an HBM budget: a request starts only when the bytes its
  plan reports (expd_plan_footprint_bytes) plus its input and output arrays
  fit beside everything already running and every cached plan; the first
  queued request (in arrival order) that fits is taken, so small requests flow
  past a large one that waits for memory;
* per-worker plan caches keyed by the full plan parameters (plans are reused
  across requests with equal parameters and evicted least recently used when
  their memory is needed).

Plans allocate stream-ordered (cudaMallocAsync / cudaFreeAsync), so creating
and destroying them does not stall the other streams.  Inputs are generated
on the device from each request's seed (u0 on the host, 8 bytes per grid
point; the separable source f = e^{-t} g(x) as a device broadcast).  Latency
is measured from a request's arrival to its result on the device.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import List, Optional

import numpy as np
import torch

from . import expd
from . import inputs as I


@dataclasses.dataclass
class Record:
    rid: int
    name: str
    arrival: float        # seconds since the trace started
    start: float
    end: float
    unknowns: int
    iterations: int
    status: int
    precision: int

    @property
    def latency(self) -> float:
        return self.end - self.arrival


# GMRES restart length of served requests: the mixed path's refinement ends a
# cycle after one or two iterations, and every basis vector of a 1024^2 x 255
# request is 2.1 GB, so the engine keeps 4 (7 vectors with the two work
# vectors; the workload default of 20 holds 23)
SERVE_GMRES_RESTART = 4


def _spec(p: I.Problem, precision: int, max_iter: int) -> expd.PlanSpec:
    return expd.spec_from_problem(p, precision=precision, max_iter=max_iter, gmres_restart=SERVE_GMRES_RESTART)


def _key(spec: expd.PlanSpec):
    return dataclasses.astuple(spec)


def request_bytes(p: I.Problem, precision: int, max_iter: int = 200) -> int:
    """Device bytes a request holds while it runs: its plan, u0, f and U."""
    spec = _spec(p, precision, max_iter)
    flags = expd.FOOTPRINT_SOURCE if p.forcing else 0
    if p.solver == "gmres":
        flags |= expd.FOOTPRINT_GMRES
    io = 8 * p.M * (1 + p.Nt * (2 if p.forcing else 1))
    return expd.plan_footprint_bytes(spec, flags) + io


def device_inputs(p: I.Problem, dev: torch.device, stream: torch.cuda.Stream):
    """u0 and f of a request on the device (f built there from its separable form)."""
    u0 = torch.from_numpy(I.make_u0(p)).to(dev, non_blocking=False)
    f = None
    if p.forcing:
        g = I.make_forcing(p.with_(Nt=1, dt=0.0))[0]         # e^{-0} g(x) = g(x)
        gd = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
        t = torch.arange(1, p.Nt + 1, dtype=torch.float64, device=dev) * p.dt
        f = torch.exp(-t).reshape((-1,) + (1,) * p.ndim) * gd.unsqueeze(0)
    return u0, f


class Admission:
    """HBM admission of queued requests (pure bookkeeping, no device calls).

    `push` queues a request with the bytes it needs; `take` returns the first
    queued request, in arrival order, whose bytes fit beside the running ones
    and the cached plans (or any request when nothing else holds memory), and
    counts it as running until `done`."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.queue: List = []
        self.in_use = 0
        self.cached = 0

    def push(self, item, need: int) -> None:
        self.queue.append((item, int(need)))

    def push_front(self, item, need: int) -> None:
        """Re-queue a request that has to wait (ahead of every later arrival)."""
        self.queue.insert(0, (item, int(need)))

    def take(self):
        for i, (item, need) in enumerate(self.queue):
            if self.in_use + self.cached + need <= self.budget or (self.in_use == 0 and self.cached == 0):
                del self.queue[i]
                self.in_use += need
                return item, need
        return None

    def done(self, need: int) -> None:
        self.in_use -= need


class Engine:
    """Runs a request trace with `workers` concurrent solves on one GPU."""

    def __init__(self, device: int = 0, workers: int = 4, budget_bytes: Optional[int] = None,
                 precision: int = expd.PREC_MIXED, max_iter: int = 200, cache_plans: bool = True,
                 tuner=None):
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        free, _ = torch.cuda.mem_get_info(self.dev)
        # 60 % of the free memory: the rest absorbs blocks that freed requests
        # leave in the allocators' pools (not yet reusable by another worker's
        # stream), which at 70 % made the largest requests' plan creation fail
        # and retry alone
        self.budget = int(budget_bytes if budget_bytes is not None else 0.6 * free)
        self.workers = workers
        self.precision = precision
        self.max_iter = max_iter
        self.cache_plans = cache_plans
        # autotune.Tuner: plans of shapes it has measured use its fastest
        # kernel variants (the defaults otherwise; it never measures here)
        self.tuner = tuner
        self._cv = threading.Condition()
        self._adm = Admission(self.budget)
        self._closed = False
        self.records: List[Record] = []
        self._alone: set = set()      # workers retrying a request alone after running out of memory
        self.errors: List[str] = []
        self.results: dict = {}
        self.keep_results = False
        self.retries = 0

    def _worker(self, wid: int, t0: float, caches: dict):
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(device=self.dev)
        cache: "collections.OrderedDict" = collections.OrderedDict()   # key -> (plan, bytes)
        caches[wid] = cache
        while True:
            with self._cv:
                got = None
                while True:
                    # a worker retrying alone after running out of memory: hand
                    # back every cached plan and take nothing new until it is done
                    if self._alone - {wid}:
                        while cache:
                            _, (pl, b) = cache.popitem(last=False)
                            pl.destroy()
                            self._adm.cached -= b
                        self._cv.notify_all()
                        self._cv.wait(timeout=0.05)
                        continue
                    got = self._adm.take()
                    if got is not None or (self._closed and not self._adm.queue):
                        break
                    # nothing fits: free this worker's cached plans before waiting
                    if cache and self._adm.queue:
                        _, (pl, b) = cache.popitem(last=False)
                        pl.destroy()
                        self._adm.cached -= b
                        continue
                    self._cv.wait(timeout=0.05)
                if got is None:
                    break
            (arrival, rid, p), need = got
            start = time.perf_counter() - t0
            status, iters = expd.OK, 0
            spec = _spec(p, self.precision, self.max_iter)
            key = _key(spec)
            requeue = False
            for attempt in range(3):
                plan = None
                status = expd.OK
                try:
                    with torch.cuda.stream(stream):
                        entry = cache.pop(key, None)
                        if entry is None:
                            if self.tuner is not None:
                                plan = self.tuner.plan_create(p, spec, stream)
                            else:
                                plan = expd.plan_create(spec, stream)
                            pbytes = plan.workspace_bytes()
                        else:
                            plan, pbytes = entry
                            with self._cv:
                                self._adm.cached -= pbytes
                        u0, f = device_inputs(p, self.dev, stream)
                        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=self.dev)
                        if p.solver == "gmres":
                            info = plan.solve_gmres(u0, f, U, stream=stream)
                        else:
                            info = plan.solve_fp(u0, f, U, stream=stream)
                        iters = info["iterations"]
                        stream.synchronize()
                        if self.keep_results:
                            self.results[rid] = U.cpu().numpy()
                        del u0, f, U
                        if self.cache_plans:
                            cache[key] = (plan, pbytes)
                            with self._cv:
                                self._adm.cached += pbytes
                        else:
                            plan.destroy()
                        plan = None
                    break
                except (expd.ExpdError, torch.cuda.OutOfMemoryError) as e:
                    status = e.status if isinstance(e, expd.ExpdError) else expd.ERR_OOM
                    if plan is not None:
                        plan.destroy()
                    u0 = f = U = None
                    if status != expd.ERR_OOM or attempt == 2:
                        self.errors.append(f"{p.name}: {e}")
                        break
                    # device memory held outside the budget (PyTorch's cache of
                    # earlier inputs, cached plans): release this worker's plans
                    # and retry; the last retry waits until this request is the
                    # only one running and every cached plan is gone, so a
                    # request that fits the device alone always completes
                    with self._cv:
                        while cache:
                            _, (pl, b) = cache.popitem(last=False)
                            pl.destroy()
                            self._adm.cached -= b
                        if attempt == 1:
                            if self._alone:
                                # another worker is already retrying alone: hand the
                                # request back to the head of the queue
                                requeue = True
                            else:
                                self._alone.add(wid)
                                while self._adm.in_use > need or self._adm.cached > 0:
                                    self._cv.notify_all()
                                    self._cv.wait(timeout=0.05)
                    if requeue:
                        break
                    # only this worker's stream is synchronised: another worker
                    # may be capturing a CUDA graph, which a device-wide
                    # synchronisation (or a free that implies one) would break
                    stream.synchronize()
                    try:
                        torch.cuda.empty_cache()
                    except RuntimeError:
                        pass
                    self.retries += 1
                except Exception as e:  # any other failure: recorded, never lost
                    status = expd.ERR_CUDA
                    self.errors.append(f"{p.name}: {type(e).__name__}: {e}")
                    if plan is not None:
                        try:
                            plan.destroy()
                        except Exception:
                            pass
                    break
            end = time.perf_counter() - t0
            with self._cv:
                self._alone.discard(wid)
                self._adm.done(need)
                if requeue:
                    self._adm.push_front((arrival, rid, p), need)
                    self._cv.notify_all()
                    continue
                self.records.append(Record(rid, p.name, arrival, start, end, p.unknowns, iters, status,
                                           self.precision))
                self._cv.notify_all()

    def run(self, requests: List[I.Request], realtime: bool = True, keep_results: bool = False) -> List[Record]:
        """Replays the trace (arrivals at their offsets when realtime) and waits.
        keep_results copies every solution to the host (self.results[rid])."""
        self.records, self.errors, self.results, self.retries = [], [], {}, 0
        self.keep_results = keep_results
        needs = [request_bytes(r.problem, self.precision, self.max_iter) for r in requests]
        for r, n in zip(requests, needs):
            if n > self.budget:
                raise ValueError(f"request {r.rid} needs {n} bytes, above the budget {self.budget}")
        caches: dict = {}
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(w, t0, caches), daemon=True)
                   for w in range(self.workers)]
        self._closed = False
        for th in threads:
            th.start()
        for r, n in zip(requests, needs):
            if realtime:
                delay = r.arrival_s - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            arr = r.arrival_s if realtime else 0.0
            with self._cv:
                self._adm.push((arr, r.rid, r.problem), n)
                self._cv.notify_all()
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for th in threads:
            th.join()
        for cache in caches.values():
            for pl, _ in cache.values():
                pl.destroy()
            cache.clear()
        self._adm.cached = 0
        return sorted(self.records, key=lambda rec: rec.rid)


def summary(records: List[Record], wall: Optional[float] = None) -> dict:
    """Latency percentiles (ms) and throughput (unknowns/s) of a finished trace."""
    lat = np.array([r.latency for r in records]) * 1e3
    span = wall if wall is not None else (max(r.end for r in records) - min(r.arrival for r in records))
    unk = sum(r.unknowns for r in records)
    ok = sum(1 for r in records if r.status == expd.OK)
    return {"requests": len(records), "ok": ok, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "unknowns": int(unk), "span_s": float(span), "throughput": unk / span if span > 0 else None}


def run_one_at_a_time(requests: List[I.Request], device: int = 0, precision: int = expd.PREC_FP64,
                      max_iter: int = 200, cache_plans: int = 4, cache_bytes: Optional[int] = None) -> List[Record]:
    """Baseline server: one request at a time, first come first served.

    Each request is solved alone (plan, inputs, solve, synchronise) to measure
    its service time (plans are reused across equal requests, up to
    `cache_plans` of them and `cache_bytes` of device memory -- half the free
    memory by default -- as the engine does); a single-server FIFO queue then
    gives start_i = max(arrival_i, end_{i-1}) and end_i = start_i + service_i,
    which is exactly what a one-at-a-time server does with these arrivals."""
    dev = torch.device("cuda", device)
    if cache_bytes is None:
        cache_bytes = int(0.5 * torch.cuda.mem_get_info(dev)[0])
    out = []
    prev_end = 0.0
    cache: "collections.OrderedDict" = collections.OrderedDict()   # the same plan reuse as the engine
    for r in sorted(requests, key=lambda q: q.arrival_s):
        p = r.problem
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        spec = _spec(p, precision, max_iter)
        key = _key(spec)
        plan = cache.pop(key, None)
        if plan is None:
            need = request_bytes(p, precision, max_iter)
            while cache and sum(pl.workspace_bytes() for pl in cache.values()) + need > cache_bytes:
                cache.popitem(last=False)[1].destroy()
            plan = expd.plan_create(spec)
        u0, f = device_inputs(p, dev, torch.cuda.current_stream())
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=dev)
        fn = plan.solve_gmres if p.solver == "gmres" else plan.solve_fp
        info = fn(u0, f, U)
        torch.cuda.synchronize(dev)
        service = time.perf_counter() - t0
        del u0, f, U
        cache[key] = plan
        while len(cache) > cache_plans:
            cache.popitem(last=False)[1].destroy()
        start = max(r.arrival_s, prev_end)
        prev_end = start + service
        out.append(Record(r.rid, p.name, r.arrival_s, start, prev_end, p.unknowns, info["iterations"], expd.OK,
                          precision))
    for pl in cache.values():
        pl.destroy()
    return sorted(out, key=lambda rec: rec.rid)


def with_rate(requests: List[I.Request], rate_per_s: float, seed: int = 5) -> List[I.Request]:
    """The same requests with seeded Poisson arrivals at `rate_per_s`."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate_per_s, size=len(requests))
    t = np.cumsum(gaps)
    return [I.Request(r.rid, float(t[i]), r.problem) for i, r in enumerate(requests)]
