"""CPU checks of the batched autotuner's host logic (paper_2105_00115_gb300/
tune.py): the cache key of a batch shape, the JSON cache written atomically
and read back, a damaged cache read as empty, and a cache hit that returns
the stored launch shape without launching anything."""
import json

import pytest

from paper_2105_00115_gb300 import tune


def test_shape_key_buckets_by_powers_of_two():
    k = tune.shape_key("GB300", 32, [256, 1 << 20, 3000])
    assert k == "GB300|B=32|count=3|total=2^20|max=2^20"
    # lengths that round to the same powers of two share a key; another block size does not
    assert tune.shape_key("GB300", 32, [250, (1 << 20) + 5, 3100]) == k
    assert tune.shape_key("GB300", 64, [256, 1 << 20, 3000]) != k
    assert tune.shape_key("GB300", 32, []) == "GB300|B=32|count=0|total=2^0|max=2^0"


def test_cache_roundtrip_and_damaged_file(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert tune._load_cache(path) == {}
    tune._store(path, "a", {"threads_per_cta": 256, "ctas_per_sm": 3, "staged": 1})
    tune._store(path, "b", {"threads_per_cta": 128, "ctas_per_sm": 6, "staged": 0})
    data = tune._load_cache(path)
    assert data["a"]["ctas_per_sm"] == 3 and data["b"]["threads_per_cta"] == 128
    assert not list((tmp_path / "sub").glob("*.tmp"))  # written through a temporary and renamed
    with open(path, "w") as fh:
        fh.write("{not json")
    assert tune._load_cache(path) == {}


def test_cache_hit_launches_nothing(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GB300")

    class FakeParams:
        block = 32

    class FakeBatch:
        p = FakeParams()
        ns_host = [256, 4096, 1 << 16]
        tuning = None

        def launch(self, stream=None):
            raise AssertionError("a cache hit must not launch")

    path = str(tmp_path / "tuning.json")
    key = tune.shape_key("GB300", 32, FakeBatch.ns_host)
    with open(path, "w") as fh:
        json.dump({key: {"threads_per_cta": 128, "ctas_per_sm": 6, "staged": 0, "times_ms": {"128x6r": 1.5}}}, fh)
    b = FakeBatch()
    tuning, times = tune.tune_batched(b, path=path)
    assert (tuning.threads_per_cta, tuning.ctas_per_sm, tuning.staged) == (128, 6, 0)
    assert b.tuning is tuning and times == {"128x6r": 1.5}
