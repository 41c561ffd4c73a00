"""The autotune cache without a GPU: keys, the JSON file, and the apply-or-tune logic with an
injected tuner (the real rk4_chain_autotune needs a GPU; the cache logic does not)."""
import json

import pytest

from paper_1412_0544_gb300 import tune_cache as tc


def test_keys_bucket_sites_and_separate_workloads():
    k = tc.make_key("NVIDIA GB300", 0, 0, 1, 1 << 24)
    assert k == tc.make_key("NVIDIA GB300", 0, 0, 1, (1 << 24) + 12345)  # same power-of-two bucket
    assert k != tc.make_key("NVIDIA GB300", 0, 0, 1, 1 << 25)
    assert k != tc.make_key("NVIDIA GB300", 0, 1, 1, 1 << 24)          # precision
    assert k != tc.make_key("NVIDIA GB300", 0, 0, 4096, 1 << 24)       # batch
    assert k != tc.make_key("NVIDIA GB300", 0, 0, 1, 1 << 24, "dopri5+nnn")
    assert k != tc.make_key("NVIDIA B200", 0, 0, 1, 1 << 24)


def test_store_and_load_round_trip(tmp_path):
    p = tmp_path / "sub" / "tune.json"
    assert tc.load(str(p)) == {}
    tc.store(str(p), "a", {"kernel": 2, "block": 256, "v": 4, "k": 1})
    tc.store(str(p), "b", {"kernel": 3, "block": 128, "v": 8, "k": 16})
    tc.store(str(p), "a", {"kernel": 2, "block": 512, "v": 4, "k": 2})
    d = json.loads(p.read_text())
    assert d == {"a": {"kernel": 2, "block": 512, "v": 4, "k": 2}, "b": {"kernel": 3, "block": 128, "v": 8, "k": 16}}
    p.write_text("{not json")
    assert tc.load(str(p)) == {}


def test_autotune_applies_cached_choice(tmp_path, monkeypatch):
    calls, applied = [], []

    def tuner():
        calls.append(1)
        return {"block": 128, "v": 8, "k": 16, "G": 896}

    kw = dict(tuner=tuner, apply=applied.append, get_kernel=lambda: 2)
    path = str(tmp_path / "t.json")
    first = tc.autotune(None, None, None, None, "key1", path=path, **kw)
    assert first["cached"] is False and first["kernel"] == 2 and len(calls) == 1 and not applied
    second = tc.autotune(None, None, None, None, "key1", path=path, **kw)
    assert second["cached"] is True and len(calls) == 1
    assert applied == [{"kernel": 2, "block": 128, "v": 8, "k": 16, "G": 896}]
    # the environment variable names the file when no path is given
    monkeypatch.setenv(tc.ENV, path)
    third = tc.autotune(None, None, None, None, "key1", **kw)
    assert third["cached"] is True and len(calls) == 1
    other = tc.autotune(None, None, None, None, "key2", **kw)
    assert other["cached"] is False and len(calls) == 2
    assert set(json.load(open(path))) == {"key1", "key2"}


def test_without_a_path_it_only_tunes(tmp_path, monkeypatch):
    monkeypatch.delenv(tc.ENV, raising=False)
    n = []
    r = tc.autotune(None, None, None, None, "k", tuner=lambda: n.append(1) or {"block": 64, "v": 1, "k": 1},
                    apply=lambda e: pytest.fail("nothing to apply"), get_kernel=lambda: 2)
    assert r["cached"] is False and n == [1]


def test_incomplete_entries_are_not_applied(tmp_path):
    path = str(tmp_path / "t.json")
    tc.store(path, "k", {"kernel": 2, "block": 256})  # no v, k
    r = tc.autotune(None, None, None, None, "k", path=path, tuner=lambda: {"block": 64, "v": 2, "k": 1},
                    apply=lambda e: pytest.fail("incomplete entry applied"), get_kernel=lambda: 2)
    assert r["cached"] is False


def test_stale_entries_are_tuned_again(tmp_path):
    """An entry the library rejects when applied (a tiling another build allowed) is replaced."""
    from paper_1412_0544_gb300 import RK4Error
    path = str(tmp_path / "t.json")
    tc.store(path, "k", {"kernel": 2, "block": 512, "v": 4, "k": 16})

    def reject(entry):
        raise RK4Error(-1, "rk4_chain_set_tiling")

    r = tc.autotune(None, None, None, None, "k", path=path, tuner=lambda: {"block": 256, "v": 4, "k": 16, "G": 896},
                    apply=reject, get_kernel=lambda: 2)
    assert r["cached"] is False and r["block"] == 256
    assert tc.load(path)["k"] == {"kernel": 2, "block": 256, "v": 4, "k": 16, "G": 896}
