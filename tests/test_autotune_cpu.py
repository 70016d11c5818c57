"""The autotuner's host logic with a model timer (no GPU): cache keys name
the device and its SM count, the coordinate descent finds the model's
optimum, results persist in the JSON cache, and circuits that fit one tile
keep the defaults without timing."""
import json

import pytest

from paper_2603_02804_gb300 import autotune as at

DEV = ("NVIDIA GB300", 152)


def model(best_K, best_rule, best_ctas):
    calls = []

    def timer(n, d, B, cfg, kind):
        calls.append((n, d, B, dict(cfg), kind))
        K = cfg["tile_bits"] or 12
        t = 10.0 + abs(K - best_K)
        t += 0.0 if cfg["catch_up"] in (0, best_rule) and (cfg["catch_up"] == best_rule or best_rule == 0) else 0.5
        t += 0.0 if cfg["fwd_ctas"] in (0, best_ctas) and (cfg["fwd_ctas"] == best_ctas or best_ctas == 0) else 0.3
        return t
    return timer, calls


def test_bucket_shape_and_key():
    assert [at.bucket(v) for v in (1, 2, 3, 4, 5, 64, 65, 200)] == [1, 2, 4, 4, 8, 64, 128, 256]
    single = at.Autotuner(path=None, dev=DEV)
    batch = at.Autotuner(path=None, kind="batch", dev=DEV)
    assert single.shape(17, 150, 40) == (17, 64, 64) and single.shape(17, 20, 5) == (17, 32, 8)
    assert batch.shape(17, 150, 40) == (17, 64, 16) and batch.shape(17, 20, 5) == (17, 32, 16)
    k = at.key(*batch.shape(17, 150, 40), "batch", DEV)
    assert k == "NVIDIA GB300|sms=152|batch|n=17|d~64|B~16"
    assert at.key(*batch.shape(17, 150, 40), "batch", ("NVIDIA GB300", 148)) != k


def test_small_circuits_keep_defaults_without_timing():
    timer, calls = model(9, 1, 3)
    t = at.Autotuner(path=None, timer=timer, dev=DEV)
    assert t.choose(12, 50, 8) == at.DEFAULT
    assert calls == []


@pytest.mark.parametrize("best", [(9, 1, 3), (12, 2, 2), (7, 2, 0)])
def test_coordinate_descent_finds_the_model_optimum(best):
    timer, calls = model(*best)
    t = at.Autotuner(path=None, timer=timer, dev=DEV)
    cfg = t.choose(16, 100, 128)
    assert (cfg["tile_bits"] or 12) == best[0]
    assert cfg["catch_up"] == best[1] or (best[1] == 0 and cfg["catch_up"] == 0)
    assert cfg["fwd_ctas"] == best[2] or (best[2] == 0 and cfg["fwd_ctas"] == 0)
    # timed on the bucketed shape, capped at depth 64 and batch 64
    assert all(c[1] == 64 and c[2] == 64 and c[0] == 16 for c in calls)
    # default + 5 widths + 2 rules + 2 instances, no configuration timed twice
    assert len(calls) == 10 and t.trials == 10
    assert len({json.dumps(c[3], sort_keys=True) for c in calls}) == 10


def test_batch_kind_does_not_tune_the_forward_instance():
    timer, calls = model(10, 1, 3)
    t = at.Autotuner(path=None, kind="batch", timer=timer, dev=DEV)
    cfg = t.choose(14, 30, 5)
    assert cfg["fwd_ctas"] == 0 and all(c[4] == "batch" and c[2] == 16 for c in calls)
    assert len(calls) == 8
    t.choose(14, 17, 60)  # the same timed shape: from the cache
    assert len(calls) == 8


def test_refused_configurations_are_skipped():
    def timer(n, d, B, cfg, kind):
        if cfg["tile_bits"] in (7, 8):
            raise RuntimeError("planner refuses")
        return 5.0 if cfg["tile_bits"] == 8 else 6.0 + (cfg["tile_bits"] or 12) * 0.01
    t = at.Autotuner(path=None, timer=timer, dev=DEV)
    assert t.choose(13, 10, 2)["tile_bits"] == 9


def test_cache_persists_and_is_keyed_by_sm_count(tmp_path):
    path = str(tmp_path / "tune.json")
    timer, calls = model(10, 2, 2)
    t1 = at.Autotuner(path=path, timer=timer, dev=DEV)
    c1 = t1.choose(15, 40, 16)
    n1 = len(calls)
    t2 = at.Autotuner(path=path, timer=timer, dev=DEV)
    assert t2.choose(15, 40, 16) == c1 and len(calls) == n1  # from the file, nothing timed
    assert t2.choose(15, 33, 9) == c1 and len(calls) == n1   # same buckets
    t3 = at.Autotuner(path=path, timer=timer, dev=("NVIDIA GB300", 148))
    t3.choose(15, 40, 16)
    assert len(calls) > n1                                     # another SM count: tuned again
    with open(path) as f:
        assert len(json.load(f)) == 2
