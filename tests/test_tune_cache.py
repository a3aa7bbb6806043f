"""Host logic of the autotuner's cache (paper_1612_09001_gb300/tune.py): shapes
stored per GPU name and model are installed again by apply_cached; a missing or
corrupt cache file installs nothing.  Runs on the CPU with a stand-in filter."""
import json

import pytest

pytest.importorskip("torch")
from paper_1612_09001_gb300 import tune  # noqa: E402


class FakeFilter:
    def __init__(self, P, Q, M):
        self.P, self.Q, self.M = P, Q, M
        self.fwd = None
        self.adj = None

    def set_fwd_launch(self, **kw):
        self.fwd = kw

    def set_adj_launch(self, gh_blocks, tap_group):
        self.adj = (gh_blocks, tap_group)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setattr(tune, "CACHE", str(path))
    monkeypatch.setattr(tune.torch.cuda, "get_device_name", lambda *a, **k: "GB300-test")
    return path


def test_store_then_apply_cached(cache):
    fwd = dict(mode=3, V=8, warps=12, stages=3, ctas_per_sm=0, use_tma=1)
    tune._store(tune._key("fwd", 9, 9, 4), fwd)
    tune._store(tune._key("adj", 9, 9, 4), [152, 5])
    assert json.loads(cache.read_text()) == {"GB300-test|fwd|P9Q9M4": fwd, "GB300-test|adj|P9Q9M4": [152, 5]}
    f = FakeFilter(9, 9, 4)
    assert tune.apply_cached(f)
    assert f.fwd == fwd and f.adj == (152, 5)
    other = FakeFilter(7, 7, 3)   # another model: nothing cached
    assert not tune.apply_cached(other)
    assert other.fwd is None and other.adj is None


def test_missing_or_corrupt_cache_installs_nothing(cache):
    f = FakeFilter(5, 5, 2)
    assert not tune.apply_cached(f)
    cache.parent.mkdir(parents=True)
    cache.write_text("{not json")
    assert not tune.apply_cached(f)
    tune._store(tune._key("fwd", 5, 5, 2), dict(mode=2, V=4, warps=8, stages=4, ctas_per_sm=0, use_tma=1))
    assert tune.apply_cached(f) and f.fwd["mode"] == 2
