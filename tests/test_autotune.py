"""Autotuner host logic (no GPU): which switches apply, candidate sets, the
choice of the fastest, the switch environment and the JSON table."""
import os
import threading

import pytest

from paper_2603_04350_gb300 import autotune as A
from paper_2603_04350_gb300 import expd
from paper_2603_04350_gb300 import inputs as I

AC = I.ALLEN_CAHN_256.with_(n=(64, 64), Nt=16)      # periodic, s = 1: 16 unknown slices
HD = I.HEAT_DIRICHLET_1024                           # Dirichlet 1024^2 (dense sine transforms)


def test_knobs_for_each_kind():
    assert A.knobs_for(AC, expd.PREC_MIXED) == ["fft", "time"]
    assert A.knobs_for(AC, expd.PREC_FP64) == ["fft"]                 # no register kernel in float64
    assert A.knobs_for(AC.with_(Nt=20), expd.PREC_MIXED) == ["fft"]   # 20 slices: shared-memory kernel only
    assert A.knobs_for(HD, expd.PREC_MIXED) == ["dst"]
    assert A.knobs_for(HD, expd.PREC_FP64) == []
    assert A.knobs_for(HD.with_(n=(1023, 1023)), expd.PREC_MIXED) == []  # fast sine transforms
    assert A.knobs_for(HD.with_(n=(1024, 1000)), expd.PREC_MIXED) == []  # not a multiple of 128


def test_candidates_are_the_product():
    c = A.candidates(AC, expd.PREC_MIXED)
    assert len(c) == 4
    flags = [f for _, f in c]
    assert 0 in flags and (expd.KF_FFT_RADIX4 | expd.KF_TIME_SMEM) in flags
    assert A.candidates(HD, expd.PREC_FP64) == [({}, 0)]


def test_tuner_picks_fastest_and_caches():
    calls = []

    def fake(p, prec, solver, flags):
        calls.append(flags)
        return 1.0 + (0.5 if flags & expd.KF_FFT_RADIX4 else 0.0) - (0.25 if flags & expd.KF_TIME_SMEM else 0.0)

    t = A.Tuner(measure=fake)
    assert t.lookup(AC, expd.PREC_MIXED) is None
    flags = t.best(AC, expd.PREC_MIXED)
    assert flags == expd.KF_TIME_SMEM and len(calls) == 4
    assert t.best(AC, expd.PREC_MIXED) == flags and len(calls) == 4        # cached
    assert t.lookup(AC.with_(Nt=32), expd.PREC_MIXED) is None             # another shape
    e = t.table[A.shape_key(AC, expd.PREC_MIXED, "fp")]
    assert e["ms"] == 0.75 and len(e["trials"]) == 4 and e["choice"] == {"fft": "four_step", "time": "smem"}


def test_table_roundtrip_and_validation(tmp_path):
    t = A.Tuner(measure=lambda p, prec, solver, flags: 2.0 if flags else 1.0)
    t.tune(HD, expd.PREC_MIXED)
    path = os.path.join(tmp_path, "tune.json")
    t.save(path)
    u = A.Tuner(measure=lambda *a: pytest.fail("must not measure"))
    u.load(path)
    assert u.lookup(HD, expd.PREC_MIXED) == 0
    for bad in ('{"k": {"env": {"LD_PRELOAD": "x"}}}', '{"k": {"flags": 64}}', '{"k": {"flags": true}}'):
        with open(path, "w") as fh:
            fh.write(bad)
        with pytest.raises(ValueError):
            u.load(path)


def test_variants_travel_as_plan_flags_not_environment(monkeypatch):
    # the tuned choice reaches the library through the scheme's kernel_flags
    # bits of each plan: the process environment is never written, so plans
    # created concurrently elsewhere are unaffected
    for k in ("EXPD_FFT_KERNEL", "EXPD_TIME_KERNEL", "EXPD_DST_TC"):
        monkeypatch.delenv(k, raising=False)
    spec = expd.spec_from_problem(AC, precision=expd.PREC_MIXED)
    tuned = A.with_flags(spec, expd.KF_TIME_SMEM | expd.KF_DST_FP64)
    assert tuned.kernel_flags == expd.KF_TIME_SMEM | expd.KF_DST_FP64
    assert spec.kernel_flags == 0 and A.with_flags(spec, None).kernel_flags == 0
    g, o, s = expd._structs(tuned)
    assert s.kernel_flags == tuned.kernel_flags
    assert not any(k in os.environ for k in ("EXPD_FFT_KERNEL", "EXPD_TIME_KERNEL", "EXPD_DST_TC"))


def test_tuner_is_thread_safe():
    t = A.Tuner(measure=lambda p, prec, solver, flags: 1.0 + flags)
    errs = []

    def worker(i):
        try:
            q = AC.with_(Nt=16 + (i % 4))
            t.tune(q, expd.PREC_MIXED)
            assert t.lookup(q, expd.PREC_MIXED) is not None
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(16)]
    for th in ts:
        th.start()
    for th in ts:
        th.join()
    assert not errs and len(t.table) == 4
