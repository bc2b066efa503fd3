"""Served mix on the GPU: concurrent solves give exactly the results of the
same requests solved alone, and meet the tolerance against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd, serve
    return expd, serve


def small_mix(count=24):
    # the mix's recipe with small grids and windows (every kind, order and a
    # ragged spread of sizes), arrivals 2 ms apart on average
    return I.served_mix(count=count, seed=7, rate_per_s=500.0, grids=(16, 32, 64), nts=(16, 32),
                        orders=(1, 2, 6))


def test_mix_results_equal_alone(mods):
    expd, serve = mods
    reqs = small_mix()
    eng = serve.Engine(workers=3, budget_bytes=2 << 30, precision=expd.PREC_MIXED)
    recs = eng.run(reqs, realtime=True, keep_results=True)
    assert not eng.errors, eng.errors
    assert len(recs) == len(reqs) and all(r.status == expd.OK for r in recs)
    for r in reqs:
        p = r.problem
        with expd.plan_create(serve._spec(p, expd.PREC_MIXED, 200)) as plan:
            u0, f = serve.device_inputs(p, DEV, torch.cuda.current_stream())
            U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
            (plan.solve_gmres if p.solver == "gmres" else plan.solve_fp)(u0, f, U)
            alone = U.cpu().numpy()
        assert np.array_equal(eng.results[r.rid], alone), p.name
        u0h, fh = I.make_inputs(p)
        ref = O.sequential_solve(O.spec_of(p), u0h, fh)[1:]
        assert O.rel_error(alone, ref) < 10 * p.tol, p.name
    s = serve.summary(recs)
    assert s["requests"] == len(reqs) and s["ok"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_tight_budget_serialises_but_completes(mods):
    expd, serve = mods
    reqs = small_mix(10)
    need = max(serve.request_bytes(r.problem, expd.PREC_MIXED) for r in reqs)
    eng = serve.Engine(workers=4, budget_bytes=need, precision=expd.PREC_MIXED)
    recs = eng.run(reqs, realtime=False)
    assert all(r.status == expd.OK for r in recs) and not eng.errors
    # whenever a request starts, the requests running then fit the budget together
    needs = {r.rid: serve.request_bytes(r.problem, expd.PREC_MIXED) for r in reqs}
    for r in recs:
        running = [q for q in recs if q.start <= r.start < q.end]
        assert sum(needs[q.rid] for q in running) <= need


def test_one_at_a_time_baseline(mods):
    expd, serve = mods
    reqs = small_mix(6)
    recs = serve.run_one_at_a_time(reqs)
    assert [r.rid for r in recs] == [r.rid for r in reqs]
    ends = [r.end for r in sorted(recs, key=lambda q: q.arrival)]
    assert all(b > a for a, b in zip(ends, ends[1:]))
    assert all(r.start >= r.arrival for r in recs)
