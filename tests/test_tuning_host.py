"""Host logic of the autotuner (no GPU): the candidate sets, the workload signature and
the JSON cache."""
import json

from paper_2411_19901_gb300 import tune


def test_candidate_sets():
    full = tune.candidates(True, "mg", 8)
    assert len(full) == 18 and len({json.dumps(c, sort_keys=True) for c in full}) == 18
    assert {c["lane_threads"] for c in full} == {64, 128, 256}
    assert {c["serial_hubs"] for c in full} == {0, 1}
    assert {c["window"] for c in full} == set(tune.WINDOWS)
    assert tune.candidates(False, "bm", 1) == tune.candidates(True, "bm", 1)
    # other k: only the default CTA size is built
    assert {c["lane_threads"] for c in tune.candidates(True, "mg", 16)} == {128}
    assert tune.candidates(True, "exact", 1) == [{}]


def test_signature_buckets_sizes():
    a = tune.signature("graph", 2**26, 1_447_511_164, True, "mg", 8)
    b = tune.signature("graph", 2**26 + 5, 1_400_000_000, True, "mg", 8)
    assert a == b
    assert a != tune.signature("graph", 2**26, 1_447_511_164, False, "mg", 8)
    assert a != tune.signature("batch", 2**26, 1_447_511_164, True, "mg", 8, count=4096)


def test_cache_round_trip(tmp_path):
    cache = str(tmp_path / "t.json")
    tune._store(cache, "k1", {"window": 8192}, [{"tuning": {"window": 8192}, "ms": 1.5}])
    tune._store(cache, "k2", {"window": 4096}, [])
    data = tune._load(cache)
    assert data["k1"]["best"] == {"window": 8192} and data["k2"]["best"] == {"window": 4096}
