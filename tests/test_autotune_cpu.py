"""Host logic of the schedule autotuner: candidate selection, shape-class keys and the
JSON cache (the timing itself runs on the GPU, in test_gpu_parity)."""
import json

import pytest

from paper_2207_03803_gb300 import autotune


def test_choose_takes_the_fastest_successful_candidate():
    times = {2: 5.0, 4: 3.0, 8: None}
    best, ms, trials = autotune.choose([{"batch_lanes": n} for n in (2, 4, 8)],
                                       lambda o: times[o["batch_lanes"]])
    assert best == {"batch_lanes": 4} and ms == 3.0
    assert [t["ms"] for t in trials] == [5.0, 3.0, None]


def test_choose_prefers_the_first_of_equal_times_and_fails_when_nothing_ran():
    best, _, _ = autotune.choose([{"a": 1}, {"a": 2}], lambda o: 1.0)
    assert best == {"a": 1}
    with pytest.raises(RuntimeError):
        autotune.choose([{"a": 1}], lambda o: None)


def test_keys_bucket_by_powers_of_two():
    k1 = autotune.fit_key("GB300", "mixed_bf16", 441968, 4000, 512)
    k2 = autotune.fit_key("GB300", "mixed_bf16", 450000, 4100, 512)
    k3 = autotune.fit_key("GB300", "mixed_bf16", 441968, 4000, 256)
    assert k1 == k2 and k1 != k3
    assert autotune.batch_key("GB300", "mixed_tf32", [1000, 3000], [200, 900]) != \
        autotune.batch_key("GB300", "mixed_tf32", [1000, 3000, 5000], [200, 900, 900])


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    c = autotune.TuneCache(path)
    assert c.get("k") is None
    c.put("k", {"batch_lanes": 4}, 3.0, [{"options": {"batch_lanes": 4}, "ms": 3.0}])
    assert autotune.TuneCache(path).get("k") == {"batch_lanes": 4}
    assert json.load(open(path))["k"]["ms"] == 3.0
