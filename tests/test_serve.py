"""Served-mix host logic: the request recipe and HBM admission (CPU only)."""
import numpy as np
import pytest

from paper_2603_04350_gb300 import inputs as I


def _serve():
    # the admission bookkeeping is plain Python; importing serve needs torch only
    from paper_2603_04350_gb300 import serve
    return serve


def test_mix_recipe():
    reqs = I.served_mix(count=400, seed=5)
    assert len(reqs) == 400
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1.0 / 100.0) < 0.002          # Poisson, 100 requests/s
    kinds = {r.problem.bc for r in reqs}
    assert kinds == {I.PERIODIC, I.DIRICHLET}
    for r in reqs:
        p = r.problem
        assert p.Ns >= p.order + 1
        if p.bc == I.DIRICHLET:
            n = p.n[0]
            # g x g interior points, the 1024^2 Dirichlet workload's solver and tolerance
            assert n in (64, 128, 256, 512, 1024) and p.n[1] == n
            assert p.forcing and p.nonlin == I.NL_NONE and p.solver == "gmres" and p.tol == 1e-9
        else:
            assert p.nonlin == I.NL_ALLEN_CAHN and (p.n[0] & (p.n[0] - 1)) == 0
    assert len({r.problem.seed for r in reqs}) == 400
    # reproducible
    again = I.served_mix(count=400, seed=5)
    assert [r.problem for r in again] == [r.problem for r in reqs]


def test_rate_rescaling_keeps_requests():
    serve = _serve()
    reqs = I.served_mix(count=300, seed=5)
    fast = serve.with_rate(reqs, 1000.0)
    assert [r.problem for r in fast] == [r.problem for r in reqs]
    assert abs(np.mean(np.diff([r.arrival_s for r in fast])) - 1e-3) < 2e-4


def test_admission_respects_budget_and_lets_small_requests_pass():
    serve = _serve()
    a = serve.Admission(100)
    for name, need in (("a", 60), ("b", 50), ("c", 30), ("d", 10)):
        a.push(name, need)
    got = [a.take() for _ in range(4)]
    # a (60) fits; b (50) does not beside it; c (30) and d (10) do
    assert got[0] == ("a", 60) and got[1] == ("c", 30) and got[2] == ("d", 10) and got[3] is None
    assert a.in_use == 100
    a.done(10)
    assert a.take() is None            # b needs 50, 10 free
    a.done(60)
    assert a.take() == ("b", 50)       # 30 running + 50
    assert a.in_use == 80


def test_admission_counts_cached_plans_and_runs_oversized_alone():
    serve = _serve()
    a = serve.Admission(100)
    a.cached = 70
    a.push("x", 40)
    assert a.take() is None            # 70 cached + 40 > 100: the caller must evict
    a.cached = 0
    a.push("huge", 500)
    assert a.take() == ("x", 40)
    assert a.take() is None            # huge waits while x runs
    a.done(40)
    assert a.take() == ("huge", 500)   # nothing else holds memory: it runs alone


def test_admission_never_exceeds_budget_random():
    serve = _serve()
    rng = np.random.default_rng(0)
    a = serve.Admission(1000)
    running = []
    for step in range(2000):
        if rng.random() < 0.6:
            a.push(step, int(rng.integers(1, 400)))
        got = a.take()
        if got is not None:
            running.append(got[1])
        assert a.in_use <= 1000 or len(running) == 1
        if running and rng.random() < 0.5:
            a.done(running.pop(int(rng.integers(0, len(running)))))


def test_admission_push_front_goes_first():
    serve = _serve()
    a = serve.Admission(100)
    a.push("late", 10)
    a.push_front("retry", 10)
    assert a.take() == ("retry", 10) and a.take() == ("late", 10)
