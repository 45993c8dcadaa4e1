"""Host logic of the autotuner (no GPU): the search, the count check, the
cache and the candidate values."""
import math

import pytest

from paper_1801_00338_gb300 import autotune as A

SIG = {"nU": 1000, "nV": 5000, "m": 50000, "side": 0, "sq_start": 10 ** 9, "sq_mid": 10 ** 7, "W": 10 ** 8}
INFO = {"auto_hubs": 1024, "auto_tau": 40, "nS": 1000 * 128}


def fake_measure(best: dict, counts=(7, 7, 28), log=None):
    """Time = number of settings that differ from `best` (+1); counts fixed."""
    def measure(t):
        if log is not None:
            log.append(dict(t))
        ms = 1.0 + sum(1.0 for k in best if t.get(k, A.DEFAULT[k]) != best[k])
        return ms, counts
    return measure


def test_descent_finds_the_separable_minimum():
    target = {"warp_max_wedges": 128, "small_max_segs": 64, "hubs": 2048, "tau": 20, "local_sweep": 1,
              "flat_max_avg": 32, "hl_max_light": 1024}
    best, ms, tried, counts = A.coordinate_descent(fake_measure(target), A.knobs_for(("exact", "local")),
                                                   dict(A.DEFAULT), INFO)
    assert best == target and ms == 1.0
    assert tried[0] == (A.DEFAULT, 8.0)
    assert counts == (7, 7, 28)


def test_descent_only_touches_the_workloads_settings():
    log = []
    A.coordinate_descent(fake_measure(dict(A.DEFAULT), log=log), A.knobs_for(("local",)), dict(A.DEFAULT), INFO)
    assert all(t["hubs"] == 0 and t["tau"] == 0 for t in log)
    assert any(t["local_sweep"] == 1 for t in log)


def test_a_setting_that_changes_a_count_is_rejected():
    def measure(t):
        return 1.0, (5,) if t["small_max_segs"] != 64 else (6,)
    with pytest.raises(RuntimeError, match="counts differ"):
        A.coordinate_descent(measure, ["small_max_segs"], dict(A.DEFAULT), INFO)


def test_hub_candidates_are_whole_tiles_within_bounds():
    vals = A.candidates("hubs", A.DEFAULT, {"auto_hubs": 3584, "nS": 10000})
    assert vals[0] == 0 and vals[1] == A.NO_HUBS
    for h in vals[2:]:
        assert h % 128 == 0 and 128 <= h <= min(16384, 10000)
    assert 1792 in vals and 7168 in vals and 14336 not in vals  # 4 x 3584 > 10000 // 128 * 128
    assert A.candidates("hubs", A.DEFAULT, {"auto_hubs": 0, "nS": 10 ** 6}) == [0, A.NO_HUBS]
    assert A.candidates("tau", A.DEFAULT, {"auto_tau": 3}) == [0, 6]
    assert A.candidates("tau", A.DEFAULT, {"auto_tau": 0}) == [0]
    assert A.candidates("tau", A.DEFAULT, {"auto_tau": 61}) == [0, 30, 122]


def test_cache_round_trip_and_reuse(tmp_path):
    path = str(tmp_path / "t.json")
    target = {"warp_max_wedges": 256, "small_max_segs": 64, "hubs": 0, "tau": 0, "local_sweep": 1, "flat_max_avg": 64,
              "hl_max_light": 0}
    log = []
    r1 = A.tune(fake_measure(target, log=log), "GB300", SIG, INFO, ("exact", "local"), path)
    assert r1.source == "search" and r1.tuning == target and r1.default_ms == 4.0
    n_search = len(log)
    assert n_search > 5
    log.clear()
    r2 = A.tune(fake_measure(target, log=log), "GB300", SIG, INFO, ("exact", "local"), path)
    assert r2.source == "cache" and r2.tuning == target
    assert len(log) == 2  # the cached choice and the default, timed once each
    # another GPU or workload does not reuse it
    log.clear()
    r3 = A.tune(fake_measure(target, log=log), "B200", SIG, INFO, ("exact", "local"), path)
    assert r3.source == "search"
    r4 = A.tune(fake_measure(target), "GB300", SIG, INFO, ("exact",), path)
    assert r4.source == "search"


def test_near_graph_starts_from_the_cached_choice(tmp_path):
    path = str(tmp_path / "t.json")
    target = {"warp_max_wedges": 256, "small_max_segs": 64, "hubs": 2048, "tau": 0, "local_sweep": 0,
              "flat_max_avg": 64, "hl_max_light": 0}
    A.tune(fake_measure(target), "GB300", SIG, INFO, ("exact", "local"), path)
    near = dict(SIG, m=int(SIG["m"] * 1.1))
    log = []
    r = A.tune(fake_measure(target, log=log), "GB300", near, INFO, ("exact", "local"), path)
    assert r.source == "search from a near graph"
    assert log[0] == target  # the first point timed is the near graph's choice
    far = dict(SIG, m=SIG["m"] * 4)
    assert A.distance(SIG, far) > A.NEAR
    assert A.lookup(A.load_cache(path), "GB300", far, ["exact", "local"]) == (None, None)
    assert A.distance(SIG, dict(SIG, side=1)) == math.inf


def test_cache_file_errors_are_tolerated(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("not json")
    assert A.load_cache(str(p)) == {}
    assert A.load_cache(str(tmp_path / "missing.json")) == {}


def test_signature_follows_the_start_side():
    st = {"nU": 10, "nV": 20, "m": 30, "sq_u": 400, "sq_v": 90, "wedges_u": 11, "wedges_v": 13}
    s0 = A.signature(st, 0)
    s1 = A.signature(st, 1)
    assert (s0["sq_start"], s0["sq_mid"], s0["W"]) == (400, 90, 13)
    assert (s1["sq_start"], s1["sq_mid"], s1["W"]) == (90, 400, 11)
