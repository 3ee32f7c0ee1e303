"""Host logic of the autotuner (no GPU): candidate selection, the JSON cache and
its key, shapes the GPU rejects.  The timing and the handle are stand-ins."""
import json

import pytest

from paper_1503_04500_gb300 import autotune, rsai


class FakeHandle:
    n = 262144

    def __init__(self, reject=()):
        self.calls = []
        self.reject = set(reject)

    def set_tuning(self, **t):
        if t["warp_bin_warps"] in self.reject:
            raise rsai.RSAIError(1, "rsai_set_tuning")
        self.calls.append(dict(t))


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(autotune, "signature", lambda n, nnz, prec: f"GB300|{prec}|n{n}|nnz{nnz}")
    cost = {(2, 0): 9.0, (2, 16): 8.0, (4, 0): 7.0, (4, 16): 5.0, (8, 0): 6.0, (8, 16): 5.5}

    def fake_time(handle, steps):
        t = handle.calls[-1]
        return cost[(t["warp_bin_warps"], t["small_qr_max_p"])]

    monkeypatch.setattr(autotune, "_time_rebuild", fake_time)
    return [dict(warp_bin_warps=w, warp_bin_ctas_per_sm=0, small_qr_max_p=sp, global_bin_ctas=0)
            for w in (2, 4, 8) for sp in (0, 16)]


def test_picks_the_fastest_and_caches_it(tmp_path, fake_gpu):
    path = str(tmp_path / "tuning.json")
    h = FakeHandle()
    r = autotune.tune(h, 1810432, "fp32_refine", candidates=fake_gpu, path=path)
    assert not r["cached"] and r["ms"] == 5.0
    assert r["tuning"]["warp_bin_warps"] == 4 and r["tuning"]["small_qr_max_p"] == 16
    assert h.calls[-1] == r["tuning"]  # the handle is left on the winner
    assert len(r["trials"]) == len(fake_gpu)
    data = json.load(open(path))
    assert list(data) == ["GB300|fp32_refine|n262144|nnz1810432"]
    # a second handle of the same signature takes the cached shape without timing
    h2 = FakeHandle()
    r2 = autotune.tune(h2, 1810432, "fp32_refine", candidates=fake_gpu, path=path)
    assert r2["cached"] and h2.calls == [r["tuning"]]
    # another precision is another key
    r3 = autotune.tune(FakeHandle(), 1810432, "fp64", candidates=fake_gpu, path=path)
    assert not r3["cached"] and len(json.load(open(path))) == 2


def test_rejected_shapes_are_skipped(tmp_path, fake_gpu):
    h = FakeHandle(reject={4})
    r = autotune.tune(h, 100, "fp64", candidates=fake_gpu, path=str(tmp_path / "t.json"))
    assert r["tuning"]["warp_bin_warps"] == 8 and r["ms"] == 5.5
    assert len(r["trials"]) == 4


def test_unreadable_cache_is_rebuilt(tmp_path, fake_gpu):
    path = tmp_path / "t.json"
    path.write_text("{ not json")
    r = autotune.tune(FakeHandle(), 100, "fp64", candidates=fake_gpu, path=str(path))
    assert not r["cached"]
    assert "GB300|fp64|n262144|nnz100" in json.load(open(path))


def test_use_cache_false_retimes(tmp_path, fake_gpu):
    path = str(tmp_path / "t.json")
    autotune.tune(FakeHandle(), 100, "fp64", candidates=fake_gpu, path=path)
    r = autotune.tune(FakeHandle(), 100, "fp64", candidates=fake_gpu, path=path, use_cache=False)
    assert not r["cached"]
