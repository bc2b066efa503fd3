#!/usr/bin/env python
"""Exp-ParaDiag benchmark: space-time unknowns per second to the workload's
relative error, mixed-precision path against the plain float64 GPU path.

Headline workload (one "step" = one whole solve of one batch of synthetic
input): 2D heat u_t = Lap u + f with homogeneous Dirichlet boundaries, the
5-point Laplacian on 1024 x 1024 interior points of (0,1)^2, Nt = 128 steps to
T = 0.1, the second-order exponential scheme (s = 2, 127 unknown slices,
133,169,152 space-time unknowns), GMRES preconditioned with Exp-ParaDiag,
alpha = 1e-3, tol 1e-9, u0 the Gaussian bump of Sec. 7 and a seeded smooth
source e^{-t} sum_i c_i sin(p_i pi x) sin(q_i pi y).  It is the largest of the
workloads that fits one GPU.  Every step runs the whole hot path: the sine
transforms of u0 and f (split-bf16 digit products on the tensor cores), the
start-up ramp and the right-hand side f_s, the GMRES iterations (each one the
residual R_s v fused with the alpha-scaled time DFT, the shifted solves and
the inverse DFT, on the float32 preconditioner, with float64 residual
refinement), and the inverse transform of the solution.

  value       whole-job unknowns/s of the mixed path, inputs resident in HBM
              (f alone is 1.07 GB, larger than L2; L2 is also flushed by a
              256 MiB write between timed steps)
  e2e         the same through the C ABI with pinned host buffers (u0 and f
              copied in, U copied out inside every timed call)
  fp64_path   the plain float64 GPU path on the same workload (speedup)
  bicgstab    the mixed path with BiCGStab (Sec. 7, Table 2)
  gpu_sequential  the same scheme stepped one time step after another on the
              GPU in float64 (the time-stepping baseline)
  roofline    the dominant kernel class of the headline solve: algorithmic
              bytes (HBM-bound classes) or executed bf16 flops (the
              tensor-core DST) per launch over its CUDA-event time, against
              MEASURED_PEAKS.json; roofline_hbm_top / roofline_tensor give
              the largest class of each kind
  legs        the other workloads: the 1D periodic heat equation (Nx = 128,
              Nt = 32, float64 fixed point, against the exact solution too),
              the 256^2 x 64 and the 512^2 x 256 order-6 periodic Allen-Cahn
              solves, each mixed against float64 with the error against the
              oracle
  served_mix  the 2,000-request mix (Poisson arrivals at 70 % of measured
              capacity): throughput and p50/p99 latency of the concurrent
              engine, and of a float64 one-request-at-a-time server
  cpu_baseline  the CPU oracle's Exp-ParaDiag GMRES on a bounded sample of the
              headline workload, one replica per host core

Launch: python bench.py [--gpus N --steps K --warmup W] (N > 1 under torchrun:
every rank solves its own seeded problem, no collective on the data path).
--impl reference times the CPU oracle (the reference arm: the paper ships no
code) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# PyTorch allocates from the CUDA stream-ordered pool the plans use too
# (cudaMallocAsync), so the served mix's request tensors and plans share one
# pool instead of two caches that fragment device memory between them
os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "backend:cudaMallocAsync")

METRIC = "space-time unknowns/sec to 1e-8 rel. error, mixed vs FP64 GPU path; p50/p99 latency"
UNIT = "unknowns/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# float64 FMA throughput on GB300 (152 SMs x 2 FMA/clk x 2.07 GHz x 2 flop)
FP64_PEAK_TFLOPS = 1.248
# classes bound by the float64 pipe on a float64 plan
FP64_CLASSES = ("time", "fft_col", "fft_row", "dst")
# the sample of the headline workload the CPU oracle solves per replica
ORACLE_SAMPLE_N = 128
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel
# class as a fraction of its algorithmic bytes, from one ncu capture of the
# same kernel on a 512^2 x 127 Dirichlet launch (traffic grows in proportion to
# the unknowns, so the fraction carries to a full launch).  time_kernel_tc:
# the refinement residual moved 765.3 MB for 799.0 MB algorithmic (0.958), the
# identity-form operator 490.2 MB for 532.6 MB (0.920); a solve runs four of
# each kind (the right-hand side launch with the residuals), so the class is
# reported at 0.94 of its algorithmic bytes per launch.  time_kernel_real
# (the FFT-based real-column kernel, on plans without the tensor-core one):
# 775.4 / 799.0 MB and 495.5 / 532.6 MB, 0.95.  dst_mma_kernel<128, 2> (the
# tensor-core DST, first pass of the source's transform): 335.2 + 222.9 MB
# for 605.2 MB algorithmic (the digits read once, the float64 result written
# once), 0.92.  An entry is removed whenever its kernel changes after the
# capture.
NCU_TRAFFIC_FRACTION = {"time": 0.95, "time_tc": 0.94, "dst_tc": 0.92}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error checks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="heat1d,ac256,ac512",
                    help="comma list of the other workloads to run (heat1d, ac256, ac512; '' for none)")
    ap.add_argument("--mix", type=int, default=2000, metavar="R",
                    help="requests of the served mix to replay (0 skips it)")
    ap.add_argument("--mix-baseline", type=int, default=200, metavar="R",
                    help="requests of the same arrivals the float64 one-at-a-time server replays")
    ap.add_argument("--mix-workers", type=int, default=4)
    ap.add_argument("--profile-case", default=None, metavar="N,NT,PREC[,S]",
                    help="run two solves of the Allen-Cahn workload on an N x N grid with NT steps "
                         "(PREC mixed|fp64, order S: 1 with the 256^2 workload's parameters, 6 with the "
                         "512^2 one's) and exit; the target of ncu captures")
    ap.add_argument("--profile-dirichlet", default=None, metavar="N,NT[,M]",
                    help="run two mixed GMRES(M) solves of the Dirichlet heat workload on an N x N grid with NT "
                         "steps (tensor-core DST; M = 20 by default) and exit; the target of ncu captures")
    return ap.parse_args()


# ------------------------------------------------------------ profile runs ---
def profile_case(spec: str) -> int:
    """Two solves (the second one is the captured steady state) of the periodic
    Allen-Cahn workload at another size; prints nothing but the iteration counts."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd, inputs as I
    parts = spec.split(",")
    n, nt = int(parts[0]), int(parts[1])
    prec = expd.PREC_FP64 if len(parts) > 2 and parts[2] == "fp64" else expd.PREC_MIXED
    order = int(parts[3]) if len(parts) > 3 else 1
    base = I.ALLEN_CAHN_512_S6 if order == 6 else I.ALLEN_CAHN_256.with_(order=order)
    p = base.with_(n=(n, n), Nt=nt)
    u0 = torch.from_numpy(I.make_u0(p)).cuda()
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device="cuda")
    with expd.plan_create(expd.spec_from_problem(p, precision=prec)) as plan:
        for _ in range(2):
            info = plan.solve_fp(u0, None, U)
    torch.cuda.synchronize()
    print("iterations", info["iterations"], "float32 sweeps", info["fp32_iterations"])
    return 0


def profile_dirichlet(spec: str) -> int:
    """Two mixed GMRES solves of the Dirichlet heat workload at another size."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd, inputs as I
    parts = [int(v) for v in spec.split(",")]
    n, nt = parts[0], parts[1]
    restart = parts[2] if len(parts) > 2 else 20
    p = I.HEAT_DIRICHLET_1024.with_(n=(n, n), Nt=nt, dt=0.1 / nt)
    u0, f = I.make_inputs(p)
    u0d, fd = torch.from_numpy(u0).cuda(), torch.from_numpy(f).cuda()
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device="cuda")
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, max_iter=200, gmres_restart=restart)
    with expd.plan_create(spec) as plan:
        for _ in range(2):
            info = plan.solve_gmres(u0d, fd, U)
    torch.cuda.synchronize()
    print("iterations", info["iterations"])
    return 0


# ----------------------------------------------------------------- helpers ---
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def with_rank_seed(p, rank: int):
    return p.with_(seed=p.seed + 1000 * rank) if rank else p


def aggregate(total_ms: float, unknowns: int, steps: int, world: int, pg=None, device=None):
    """Whole-job timing of a weak-scaled replica run: the slowest rank's time
    (max over ranks) and the units all ranks processed in it."""
    if pg is not None:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * unknowns * steps / (total_ms / 1e3)


def config_dict(p, world, solver):
    return {"workload": p.name, "grid": list(p.n), "bc": p.bc, "Nt": p.Nt, "Ns": p.Ns, "order": p.order,
            "alpha": p.alpha, "dt": p.dt, "tol": p.tol, "nonlin": p.nonlin, "solver": solver,
            "unknowns_per_solve": p.unknowns,
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "inputs larger than L2 (f: 1.07 GB) and L2 flushed (256 MiB write) between timed steps"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return None


def hbm_peak():
    d = _peaks()
    if d and "hbm_gbs" in d:
        return float(d["hbm_gbs"]), "measured (hbm_gbs)"
    return FALLBACK_HBM_GBS, "fallback"


def bf16_peak(sustained: bool):
    """Dense bf16 tensor peak in TFLOP/s: the measured cuBLAS figure (burst for
    a kernel timed alone, sustained for one timed inside a long step)."""
    d = _peaks()
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    if d and key in d:
        return float(d[key]), f"measured ({key})"
    return (1700.0 if sustained else FALLBACK_BF16_TFLOPS), "fallback"


def kernel_table(classes):
    return {k: {"launches": v["count"], "ms_total": round(v["ms"], 4),
                "avg_us": round(1e3 * v["ms"] / v["count"], 3) if v["count"] else None,
                "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] else None,
                "GFLOPs": round(v["flops"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] else None}
            for k, v in classes.items() if v["count"]}


def roofline_of(classes, k, fp64_plan: bool, unknowns=None):
    """The roofline entry of kernel class k from per-launch CUDA-event times:
    achieved = algorithmic bytes (or flops) per launch / average launch time."""
    c = classes[k]
    n = max(c["count"], 1)
    sec = c["ms"] / n / 1e3
    if k == "dst_tc":
        # executed bf16 digit products against the dense bf16 peak; every
        # launch is timed alone by its own event pair, so the burst figure
        peak, src = bf16_peak(sustained=False)
        ach = (c["flops"] / n) / sec / 1e12
        frac_t = NCU_TRAFFIC_FRACTION.get(k)
        return {"bound": "tensor", "kernel": k, "achieved": ach, "peak": peak, "peak_source": src,
                "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": frac_t * c["bytes"] / n if frac_t is not None else None,
                "algorithmic_bytes_per_launch": c["bytes"] / n,
                "flops_per_launch": c["flops"] / n,
                "note": "bf16 digit products executed per launch (pairs x 2 rows N K)"}
    if fp64_plan and k in FP64_CLASSES:
        ach = (c["flops"] / n) / sec / 1e12
        return {"bound": "alu", "kernel": k, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "float64 FMA rate: 152 SMs x 2 FMA/clk x 2.07 GHz", "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None}
    peak, src = hbm_peak()
    ach = (c["bytes"] / n) / sec / 1e9
    frac_t = NCU_TRAFFIC_FRACTION.get(k)
    traffic = frac_t * c["bytes"] / n if frac_t is not None else None
    return {"bound": "hbm", "kernel": k, "achieved": ach, "peak": peak, "peak_source": src, "unit": "GB/s",
            "frac": ach / peak, "traffic": traffic, "algorithmic_bytes_per_launch": c["bytes"] / n}


# ------------------------------------------------------------ cpu oracle ---
def _oracle_sample():
    from paper_2603_04350_gb300 import inputs as I
    return I.HEAT_DIRICHLET_1024.with_(name=f"heat_dirichlet_{ORACLE_SAMPLE_N}x{ORACLE_SAMPLE_N}_nt128_s2",
                                       n=(ORACLE_SAMPLE_N, ORACLE_SAMPLE_N))


def _oracle_worker(_):
    """One oracle Exp-ParaDiag GMRES solve of the sample (in a worker process)."""
    import oracle as O
    from paper_2603_04350_gb300 import inputs as I
    p = _oracle_sample()
    u0, f = I.make_inputs(p)
    t0 = time.perf_counter()
    res = O.gmres(O.spec_of(p), u0, f, tol=p.tol / math.sqrt(p.Ns), restart=20)
    return time.perf_counter() - t0, res.iterations


def oracle_pool():
    """A spawn pool with one single-threaded oracle worker per host core,
    started before any CUDA call (a process forked after one would hang)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def cpu_baseline(pool, cores, rounds=1):
    """The oracle on every host core: `cores` independent replicas of the
    sample solved at once, `rounds` times; unknowns of all replicas / wall time."""
    p = _oracle_sample()
    t0 = time.perf_counter()
    res = []
    for _ in range(rounds):
        res = pool.map(_oracle_worker, range(cores))
    wall = time.perf_counter() - t0
    value = cores * rounds * p.unknowns / wall
    per = statistics.mean(t for t, _ in res)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the headline workload at {ORACLE_SAMPLE_N}^2 interior points (same Nt = 128, s = 2, "
                      f"alpha, tol, source): numpy float64 Exp-ParaDiag GMRES ({res[0][1]} iterations), one "
                      f"single-threaded replica per core, {rounds} round(s), {wall:.1f} s wall, {per:.1f} s per solve",
            "wall_s": wall}


def run_reference(args):
    """The reference arm: the oracle (the paper ships no code) on the host
    cores, every step one round of replicas of the bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    pool, cores = oracle_pool()
    p = _oracle_sample()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pool.map(_oracle_worker, range(cores))
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    pool.close()
    total = sum(times)
    value = cores * p.unknowns * len(times) / total
    from paper_2603_04350_gb300 import inputs as I
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(I.HEAT_DIRICHLET_1024, 1, "gmres"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"every step: {cores} single-threaded replicas (one per core) of the "
                                       f"headline workload at {ORACLE_SAMPLE_N}^2 interior points, numpy float64 "
                                       "Exp-ParaDiag GMRES"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm ---
class Runner:
    """Timed whole solves on one stream: CUDA events around every solve, a
    256 MiB L2 flush between them, optional per-launch event timing."""

    def __init__(self, torch, stream, flush, barrier):
        self.torch, self.stream, self.flush, self.barrier = torch, stream, flush, barrier

    def steps(self, plan, solver, u0, f, U, K, warm, timing=False):
        torch = self.torch
        fn = {"fp": plan.solve_fp, "gmres": plan.solve_gmres, "bicgstab": plan.solve_bicgstab,
              "sequential": plan.solve_sequential}[solver]
        for k in range(warm):
            self.flush.fill_(float(k))
            fn(u0, f, U)
        self.barrier()
        plan.timing_read(reset=True)
        plan.timing_enable(timing)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        infos = []
        self.barrier()
        for k in range(K):
            self.flush.fill_(float(k + 1))
            starts[k].record(self.stream)
            infos.append(fn(u0, f, U))
            ends[k].record(self.stream)
        self.barrier()
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        tm = plan.timing_read(reset=True)
        plan.timing_enable(False)
        return ms, infos, tm


def oracle_ref(p, u0, f):
    import oracle as O
    return O.sequential_solve(O.spec_of(p), u0, f)[1:]


def errs(U, ref):
    """Sec. 7's error norm and the largest grid-point error of any slice
    relative to that slice's largest value."""
    import oracle as O
    d = np.abs(U - ref).reshape(U.shape[0], -1).max(axis=1)
    r = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return {"rel_error": O.rel_error(U, ref), "slice_elementwise": float((d / np.maximum(r, 1e-300)).max())}


def headline(args, run, dev, stream, world, pg, rank, check, clocks):
    torch = run.torch
    from paper_2603_04350_gb300 import expd, inputs as I
    p = with_rank_seed(I.HEAT_DIRICHLET_1024, rank)
    u0, f = I.make_inputs(p)
    u0d, fd = torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=dev)
    spec = expd.spec_from_problem(p, precision=expd.PREC_MIXED, max_iter=200)
    with expd.plan_create(spec, stream) as plan:
        clocks.start()
        ms, infos, tm_plain = run.steps(plan, "gmres", u0d, fd, U, args.steps, args.warmup)
        clk = clocks.stop()
        U_mixed = U.cpu().numpy()
        total_ms, value = aggregate(sum(ms), p.unknowns, args.steps, world, pg, dev)
        # the same solves with an event pair around every kernel launch: per-kernel
        # durations for the roofline and the kernel table (not the headline run)
        ms_ev, _, tm = run.steps(plan, "gmres", u0d, fd, U, 2, 0, timing=True)
        # end to end through the C ABI: pinned host u0, f in and U out inside the call
        u0_h = torch.from_numpy(u0).pin_memory()
        f_h = torch.from_numpy(f).pin_memory()
        U_h = torch.empty((p.Nt,) + p.n, dtype=torch.float64).pin_memory()
        plan.solve_gmres(u0_h, f_h, U_h)
        run.barrier()
        e2e_t = []
        for k in range(max(3, args.steps // 2)):
            run.flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.solve_gmres(u0_h, f_h, U_h)     # returns after U is in host memory
            e2e_t.append(time.perf_counter() - t0)
        e2e_value = world * p.unknowns / statistics.mean(e2e_t)
        U_e2e = U_h.numpy().copy()
    # BiCGStab on the same mixed path
    with expd.plan_create(spec, stream) as plan:
        ms_bi, infos_bi, _ = run.steps(plan, "bicgstab", u0d, fd, U, 3, 1)
        U_bi = U.cpu().numpy()
    # the plain float64 path and float64 sequential stepping
    spec64 = expd.spec_from_problem(p, precision=expd.PREC_FP64, max_iter=200)
    with expd.plan_create(spec64, stream) as plan:
        ms64, infos64, _ = run.steps(plan, "gmres", u0d, fd, U, 2, 1)
        U_fp64 = U.cpu().numpy()
        ms_seq, _, _ = run.steps(plan, "sequential", u0d, fd, U, 2, 1)
        U_seq = U.cpu().numpy()
    value64 = p.unknowns / (statistics.mean(ms64) / 1e3)
    value_seq = p.unknowns / (statistics.mean(ms_seq) / 1e3)
    classes = tm["classes"]
    dom = max(classes, key=lambda k: classes[k]["ms"])
    mem = [k for k in classes if classes[k]["count"] and k != "dst_tc"]
    info = infos[-1]
    out = {
        "value": value, "ms_per_step": total_ms / args.steps, "config": config_dict(p, world, "gmres"),
        "iterations": info["iterations"], "refinements": info["refinements"],
        "residual_history": info["history"],
        "phase_ms": {"setup": info["ms_setup"], "iterate": info["ms_iterate"], "output": info["ms_output"]},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "ms_per_step_with_kernel_events": statistics.mean(ms_ev),
        "fp64_path": {"value": value64, "ms_per_step": statistics.mean(ms64),
                      "iterations": infos64[-1]["iterations"]},
        "speedup_vs_fp64": value / (world * value64),
        "bicgstab": {"value": p.unknowns / (statistics.mean(ms_bi) / 1e3), "ms_per_step": statistics.mean(ms_bi),
                     "iterations": infos_bi[-1]["iterations"], "refinements": infos_bi[-1]["refinements"]},
        "gpu_sequential": {"value": value_seq, "ms_per_step": statistics.mean(ms_seq),
                           "note": "float64 IF-BDF2 stepping in the eigenbasis, one time step after another"},
        "speedup_vs_gpu_sequential": value / (world * value_seq),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(u0.nbytes + f.nbytes),
                "d2h_bytes_per_step": int(U_h.numel() * 8)},
        "gpu_launches": int(tm_plain["launches"]),
        "roofline": roofline_of(classes, dom, fp64_plan=False, unknowns=p.unknowns),
        "roofline_hbm_top": roofline_of(classes, max(mem, key=lambda k: classes[k]["ms"]), False, p.unknowns)
        if mem else None,
        "roofline_tensor": roofline_of(classes, "dst_tc", False) if classes.get("dst_tc", {}).get("count") else None,
        "kernels": kernel_table(classes),
    }
    if clk:
        out["clocks"] = clk
    if check:
        ref = oracle_ref(p, u0, f)
        out["rel_err_vs_oracle"] = {"mixed": errs(U_mixed, ref), "e2e": errs(U_e2e, ref),
                                    "bicgstab": errs(U_bi, ref), "fp64": errs(U_fp64, ref),
                                    "gpu_sequential": errs(U_seq, ref)}
    return out


def leg(run, dev, stream, p, solver, variants, K, warm, check, exact=None):
    """One workload on each (name, precision, scheme options) variant: value,
    time per solve, iterations, the dominant kernel's roofline, the error
    against the oracle (and against an exact solution when one is given)."""
    torch = run.torch
    from paper_2603_04350_gb300 import expd, inputs as I
    u0, f = I.make_inputs(p)
    u0d = torch.from_numpy(u0).to(dev)
    fd = None if f is None else torch.from_numpy(f).to(dev)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=dev)
    out = {"workload": p.name, "unknowns": p.unknowns, "tol": p.tol, "solver": solver}
    ref = oracle_ref(p, u0, f) if check else None
    for name, prec, kw, slv in variants:
        with expd.plan_create(expd.spec_from_problem(p, precision=prec, max_iter=200, **kw), stream) as plan:
            ms, infos, _ = run.steps(plan, slv, u0d, fd, U, K, warm)
            _, _, tm = run.steps(plan, slv, u0d, fd, U, 1, 0, timing=True)
            Uh = U.cpu().numpy()
        cls = tm["classes"]
        dom = max(cls, key=lambda k: cls[k]["ms"])
        d = {"value": p.unknowns / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms),
             "launches_per_solve": int(tm["launches"]),
             "dominant_kernel": roofline_of(cls, dom, fp64_plan=(prec == expd.PREC_FP64), unknowns=p.unknowns)}
        if infos[-1] is not None:
            d["iterations"] = infos[-1]["iterations"]
            d["fp32_iterations"] = infos[-1]["fp32_iterations"]
        if ref is not None:
            d["rel_err_vs_oracle"] = errs(Uh, ref)
        if exact is not None:
            d["rel_err_vs_exact"] = errs(Uh, exact)
        out[name] = d
    if "mixed" in out and "fp64" in out:
        out["speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def heat1d_exact(p):
    """The exact solution of the 1D periodic heat workload: the spectral
    exponential Euler step reproduces e^{-k^2 t} on each Fourier mode."""
    from paper_2603_04350_gb300 import inputs as I
    x = I.grid_coords(p)[0]
    rng = np.random.default_rng(p.seed)
    ak, bk = rng.standard_normal(16), rng.standard_normal(16)
    return np.array([sum(math.exp(-k * k * (n + 1) * p.dt) * (ak[k - 1] * np.cos(k * x) + bk[k - 1] * np.sin(k * x))
                         / k ** 2 for k in range(1, 17)) for n in range(p.Nt)])


def other_legs(args, run, dev, stream, check):
    from paper_2603_04350_gb300 import expd, inputs as I
    names = [s for s in args.legs.split(",") if s]
    out = {}
    both = [("fp64", expd.PREC_FP64, {}, "fp"), ("mixed", expd.PREC_MIXED, {}, "fp")]
    if "heat1d" in names:
        p = I.HEAT1D
        out[p.name] = leg(run, dev, stream, p, "fp", both, 20, 3, check, exact=heat1d_exact(p))
    if "ac256" in names:
        p = I.ALLEN_CAHN_256
        out[p.name] = leg(run, dev, stream, p, "fp",
                          both + [("mixed_mean_jacobian", expd.PREC_MIXED, {"jacobian": expd.JAC_MEAN_U0}, "fp"),
                                  ("gpu_sequential", expd.PREC_FP64, {}, "sequential")], 10, 3, check)
    if "ac512" in names:
        p = I.ALLEN_CAHN_512_S6
        out[p.name] = leg(run, dev, stream, p, "fp", both, 3, 1, check)
    return out


def served_mix(count: int, base_count: int, workers: int, local: int) -> dict:
    """The served mix: heterogeneous requests (kind, grid, Nt, order drawn per
    request, seed 5) replayed with Poisson arrivals at 70 % of the engine's
    measured capacity; latency from arrival to result on the device.  Baseline:
    the float64 path serving one request at a time, first come first served,
    on the first base_count requests of the same arrivals."""
    from paper_2603_04350_gb300 import expd, inputs as I, serve
    reqs = I.served_mix(count=count, seed=5)
    eng = serve.Engine(device=local, workers=workers, precision=expd.PREC_MIXED)
    eng.run(reqs[: min(16, count)], realtime=False)               # warm-up: plans, kernels
    t0 = time.perf_counter()
    eng.run(reqs, realtime=False)                                  # all queued at t = 0
    cap_span = time.perf_counter() - t0
    capacity = count / cap_span
    rate = 0.7 * capacity
    timed = serve.with_rate(reqs, rate, seed=5)
    recs = eng.run(timed, realtime=True)
    mixed = serve.summary(recs)
    nb = min(base_count, count)
    base = serve.summary(serve.run_one_at_a_time(timed[:nb], device=local, precision=expd.PREC_FP64))
    mixed_first = serve.summary([r for r in recs if r.rid < nb])
    return {"requests": count, "seed": 5, "workers": workers, "capacity_req_per_s": capacity,
            "rate_per_s": rate, "mixed_concurrent": mixed,
            "mixed_concurrent_first_requests": dict(mixed_first, requests_counted=nb),
            "fp64_one_at_a_time": dict(base, requests_replayed=nb),
            "errors": eng.errors[:5], "oom_retries": eng.retries,
            "note": "grids {64..1024}^2, Nt {16..256}, s {1,2,6}, kind {Allen-Cahn periodic (fixed point, tol 1e-8), "
                    "heat Dirichlet (g x g interior points, GMRES, tol 1e-9)}; the float64 server replays the first "
                    f"{nb} requests of the same arrivals"}


def main():
    args = parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.profile_dirichlet:
        return profile_dirichlet(args.profile_dirichlet)
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    pool, cores = oracle_pool() if want_cpu else (None, 0)   # before the first CUDA call
    import torch
    import __graft_entry__ as g
    g.build()

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # a stream of its own (the legacy default stream cannot hold CUDA graphs)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    run = Runner(torch, stream, flush, barrier)
    check = rank == 0 and not args.no_check
    h = headline(args, run, dev, stream, world, pg, rank, check, ClockSampler(local))

    out = {"metric": METRIC, "value": h.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": h.pop("ms_per_step"), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
           "config": h.pop("config")}
    out.update(h)
    if rank == 0:
        out["legs"] = other_legs(args, run, dev, stream, check)
        if args.mix > 0:
            out["served_mix"] = served_mix(args.mix, args.mix_baseline, args.mix_workers, local)
    if want_cpu:
        out["cpu_baseline"] = cpu_baseline(pool, cores)
        pool.close()
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
