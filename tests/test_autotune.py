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
    envs = [e for _, e in c]
    assert {} in envs and {"EXPD_FFT_KERNEL": "radix4", "EXPD_TIME_KERNEL": "smem"} in envs
    assert A.candidates(HD, expd.PREC_FP64) == [({}, {})]


def test_tuner_picks_fastest_and_caches():
    calls = []

    def fake(p, prec, solver, env):
        calls.append(dict(env))
        return 1.0 + (0.5 if "EXPD_FFT_KERNEL" in env else 0.0) - (0.25 if "EXPD_TIME_KERNEL" in env else 0.0)

    t = A.Tuner(measure=fake)
    assert t.lookup(AC, expd.PREC_MIXED) is None
    env = t.best(AC, expd.PREC_MIXED)
    assert env == {"EXPD_TIME_KERNEL": "smem"} and len(calls) == 4
    assert t.best(AC, expd.PREC_MIXED) == env and len(calls) == 4        # cached
    assert t.lookup(AC.with_(Nt=32), expd.PREC_MIXED) is None             # another shape
    e = t.table[A.shape_key(AC, expd.PREC_MIXED, "fp")]
    assert e["ms"] == 0.75 and len(e["trials"]) == 4 and e["choice"] == {"fft": "four_step", "time": "smem"}


def test_table_roundtrip_and_validation(tmp_path):
    t = A.Tuner(measure=lambda p, prec, solver, env: 2.0 if env else 1.0)
    t.tune(HD, expd.PREC_MIXED)
    path = os.path.join(tmp_path, "tune.json")
    t.save(path)
    u = A.Tuner(measure=lambda *a: pytest.fail("must not measure"))
    u.load(path)
    assert u.lookup(HD, expd.PREC_MIXED) == {}
    with open(path, "w") as fh:
        fh.write('{"k": {"env": {"LD_PRELOAD": "x"}}}')
    with pytest.raises(ValueError):
        u.load(path)


def test_variant_env_sets_clears_and_restores(monkeypatch):
    monkeypatch.setenv("EXPD_FFT_KERNEL", "radix4")
    monkeypatch.delenv("EXPD_DST_TC", raising=False)
    with A.variant_env({"EXPD_DST_TC": "0"}):
        assert os.environ.get("EXPD_DST_TC") == "0"
        assert "EXPD_FFT_KERNEL" not in os.environ
        # the lock is held while the switches are set
        assert not A._ENV_LOCK.acquire(blocking=False)
    assert os.environ.get("EXPD_FFT_KERNEL") == "radix4"
    assert "EXPD_DST_TC" not in os.environ


def test_variant_env_serialises_threads():
    seen = []

    def worker(v):
        with A.variant_env({"EXPD_TIME_KERNEL": v}):
            seen.append(os.environ.get("EXPD_TIME_KERNEL") == v)

    ts = [threading.Thread(target=worker, args=("smem" if i % 2 else "reg",)) for i in range(16)]
    for th in ts:
        th.start()
    for th in ts:
        th.join()
    assert all(seen) and len(seen) == 16
