"""The autotuner's search logic on the CPU: the timing is replaced by a cost
function of the thresholds currently set (hs_get_tuning needs no GPU)."""
from __future__ import annotations


def test_coordinate_descent_picks_each_knobs_best(monkeypatch):
    from paper_1109_3739_gb300 import hspgemm as h
    from paper_1109_3739_gb300 import tune

    # a separable cost: the best value of each knob is known
    want = {"warp_s_max": 64, "mid_s_max": 768, "large_s_max": 4096, "sym_mid_s_max": 512,
            "sym_heavy_from": 6144, "sort_max": 512, "sort_pct": 75, "spa_max": 2048, "heavy_part_kb": 32, "num_heavy_from": 4096}

    def fake_time(run, trials, stream=None):
        t = h.get_tuning()
        return 10.0 + sum(abs(t[k] - v) / 1000.0 for k, v in want.items())

    monkeypatch.setattr(tune, "time_ms", fake_time)
    try:
        best, log = tune.tune(lambda: None, trials=1)
        assert best == want
        assert h.get_tuning() == want            # left set
        assert log[0][0] == {"warp_s_max": 128, "mid_s_max": 1024, "large_s_max": 4096,
                             "sym_mid_s_max": 1024, "sym_heavy_from": 0, "sort_max": 1024,
                             "sort_pct": 50, "spa_max": 0, "heavy_part_kb": 16,
                             "num_heavy_from": 0}  # the defaults first
        # one timing for the defaults, then every other candidate once
        n_other = sum(len(v) - 1 for v in tune.CANDIDATES.values())
        assert len(log) == 1 + n_other
    finally:
        h.set_tuning(None)


def test_tuning_keeps_the_defaults_when_nothing_is_faster(monkeypatch):
    from paper_1109_3739_gb300 import hspgemm as h
    from paper_1109_3739_gb300 import tune
    defaults = None

    def fake_time(run, trials, stream=None):
        nonlocal defaults
        t = h.get_tuning()
        if defaults is None:
            defaults = dict(t)
        return 1.0 if t == defaults else 2.0

    monkeypatch.setattr(tune, "time_ms", fake_time)
    try:
        best, _ = tune.tune(lambda: None, trials=1)
        assert best == defaults and h.get_tuning() == defaults
    finally:
        h.set_tuning(None)


def test_work_shape_and_key():
    from paper_1109_3739_gb300 import tune
    f = [0, 10, 100, 100, 300, 5000, 20000]
    shape = tune.work_shape(f, nnz_c=20000)
    assert len(shape["bands"]) == len(tune.FLOP_BANDS)
    assert shape["bands"][0] == 0 and shape["bands"][1] == 0   # 10 of 25510 products: 0 %
    assert shape["bands"][-1] == 80                             # 20000 / 25510 = 78 % -> 80
    assert shape["c_per_flop"] == 0.8
    assert sum(shape["bands"]) in range(95, 106)
    k1 = tune.cache_key("GB300", "plus_times", "f32", shape)
    k2 = tune.cache_key("GB300", "plus_times", "f64", shape)
    assert k1 != k2 and k1 == tune.cache_key("GB300", "plus_times", "f32", dict(shape))


def test_tune_cached_times_once_per_key(monkeypatch, tmp_path):
    from paper_1109_3739_gb300 import hspgemm as h
    from paper_1109_3739_gb300 import tune
    calls = []

    def fake_time(run, trials, stream=None):
        calls.append(1)
        t = h.get_tuning()
        return 1.0 + abs(t["sort_pct"] - 75) / 100.0

    monkeypatch.setattr(tune, "time_ms", fake_time)
    path = str(tmp_path / "tuning.json")
    try:
        best, log, hit = tune.tune_cached(lambda: None, "key-a", trials=1, path=path)
        assert not hit and best["sort_pct"] == 75 and len(log) == len(calls) > 1
        n = len(calls)
        h.set_tuning(None)
        best2, log2, hit2 = tune.tune_cached(lambda: None, "key-a", trials=1, path=path)
        assert hit2 and log2 == [] and len(calls) == n and best2 == best and h.get_tuning() == best
        _, _, hit3 = tune.tune_cached(lambda: None, "key-b", trials=1, path=path)
        assert not hit3 and len(calls) > n
        import json
        assert set(json.load(open(path))) == {"key-a", "key-b"}
    finally:
        h.set_tuning(None)
