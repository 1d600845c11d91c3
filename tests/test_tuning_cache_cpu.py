"""The autotuners' JSON cache (host bookkeeping): entries are reused only for
the same library build and GPU name, the file is discarded otherwise, hits
never call the tuners, misses call them once and are stored."""
import json
from types import SimpleNamespace

import pytest

from paper_0803_1975_gb300 import gfp, tuning_cache
from paper_0803_1975_gb300.tuning_cache import TuningCache, batch_signature


@pytest.fixture
def fake_tuners(monkeypatch):
    calls = {"dot": 0, "batched": 0, "set": []}

    def dot(p, m, k, n):
        calls["dot"] += 1
        return {"word": "u32", "d": 3, "Q": 256, "kb": 60, "ms": 0.035}, []

    def batched(probs, count, workspace=None):
        calls["batched"] += 1
        return [1, 0, 4, 4, 4, -1, -1]

    monkeypatch.setattr(gfp, "gfp_dot_autotune", dot)
    monkeypatch.setattr(gfp, "gfp_batched_autotune", batched)
    monkeypatch.setattr(gfp, "gfp_batched_set_table", lambda t: calls["set"].append(list(t)))
    return calls


def probs_of(shapes):
    return [SimpleNamespace(p=p, m=m, k=k, n=n) for p, m, k, n in shapes]


def test_hits_skip_the_tuners_and_misses_are_stored(tmp_path, fake_tuners):
    path = str(tmp_path / "tune.json")
    c = TuningCache(path, stamp="abc", device="GB300")
    assert c.dot(3, 1024, 1024, 1024) == ("u32", 3, 256, 60)
    assert c.dot(3, 1024, 1024, 1024) == ("u32", 3, 256, 60)
    assert fake_tuners["dot"] == 1
    pr = probs_of([(3, 100, 100, 100), (5, 500, 500, 500), (251, 30, 30, 30)])
    assert c.batched(pr, 3) == [1, 0, 4, 4, 4, -1, -1]
    c2 = TuningCache(path, stamp="abc", device="GB300")
    assert c2.reused
    assert c2.dot(3, 1024, 1024, 1024) == ("u32", 3, 256, 60)
    assert c2.batched(pr, 3) == [1, 0, 4, 4, 4, -1, -1]
    assert fake_tuners["dot"] == 1 and fake_tuners["batched"] == 1
    assert fake_tuners["set"] == [[1, 0, 4, 4, 4, -1, -1]]


@pytest.mark.parametrize("stamp,device", [("other", "GB300"), ("abc", "B200")])
def test_stale_file_is_discarded(tmp_path, fake_tuners, stamp, device):
    path = str(tmp_path / "tune.json")
    c = TuningCache(path, stamp="abc", device="GB300")
    c.dot(5, 64, 64, 64)
    c3 = TuningCache(path, stamp=stamp, device=device)
    assert not c3.reused and c3.data["dot"] == {}
    c3.dot(5, 64, 64, 64)
    assert fake_tuners["dot"] == 2
    with open(path) as f:
        saved = json.load(f)
    assert saved["library"] == stamp and saved["device"] == device


def test_corrupt_file_is_rebuilt(tmp_path, fake_tuners):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    c = TuningCache(str(path), stamp="abc", device="GB300")
    assert not c.reused
    c.dot(3, 8, 8, 8)
    assert json.loads(path.read_text())["dot"]


def test_batch_signature_counts_buckets_and_engines():
    a = batch_signature([(3, 16, 16, 16), (3, 20, 20, 20), (251, 16, 16, 16), (5, 600, 100, 100)])
    assert a == "0h:1,0t:2,5t:1"
    assert batch_signature([(5, 600, 100, 100), (3, 20, 20, 20), (3, 16, 16, 16), (251, 16, 16, 16)]) == a


def test_library_stamp_hashes_the_file(tmp_path):
    f = tmp_path / "lib.so"
    f.write_bytes(b"abc")
    s1 = tuning_cache.library_stamp(str(f))
    f.write_bytes(b"abd")
    assert tuning_cache.library_stamp(str(f)) != s1 and len(s1) == 16
