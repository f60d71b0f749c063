"""The cache of autotuned options (paper_2111_12493_gb300.tuning), on the CPU:
shape keys, the JSON file, and that a known shape skips the tuner. The
library calls are replaced by stand-ins; tests/test_gpu_batched.py and
tests/test_gpu_parity.py run the tuner itself on a GPU."""

import json

import pytest

from paper_2111_12493_gb300 import bisim, tuning


def _stats(**kw):
    s = dict(n_vertices=1_000_000, n_edges=10_000_000, n_graphs=1, n_small=900_000, n_mid=90_000, n_hub=12)
    s.update(kw)
    return s


def test_round_to_two_significant_digits():
    assert [tuning._round2(x) for x in (0, 7, 42, 123, 1049, 1050, 987_654)] == [0, 7, 42, 120, 1000, 1100, 990_000]


def test_shape_key_separates_shapes_and_merges_near_copies():
    opts = {"direction": 0, "n_label_filter": 0, "hash_bits": 64}
    k = tuning.shape_key(_stats(), opts, "GPU A")
    assert k == tuning.shape_key(_stats(n_edges=10_040_000), opts, "GPU A")        # same two digits
    assert k != tuning.shape_key(_stats(n_edges=12_000_000), opts, "GPU A")
    assert k != tuning.shape_key(_stats(n_graphs=4096), opts, "GPU A")
    assert k != tuning.shape_key(_stats(n_hub=0), opts, "GPU A")
    assert k != tuning.shape_key(_stats(), dict(opts, direction=2), "GPU A")
    assert k != tuning.shape_key(_stats(), opts, "GPU B")


def test_cache_file_round_trip_and_version(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = tuning.TuneCache(path)
    assert c.lookup("x") is None
    want = dict(small_max_degree=16, mid_max_degree=4096, hub_chunk=2048, batch_split=0)
    c.store("x", dict(want, flags=3))                # only tuning fields are kept
    again = tuning.TuneCache(path)
    assert again.lookup("x") == want
    data = json.load(open(path))
    data["version"] = 999
    json.dump(data, open(path, "w"))
    assert tuning.TuneCache(path).lookup("x") is None  # another format: ignored


def test_known_shape_skips_the_tuner(tmp_path, monkeypatch):
    calls = {"autotune": 0, "retune": []}
    stats = _stats()
    chosen = dict(small_max_degree=8, mid_max_degree=2048, hub_chunk=1024, batch_split=0)

    def fake_autotune(ctx, rounds=2, stream=None):
        calls["autotune"] += 1
        return dict(chosen, k_incremental=2, hash_bits=64)

    monkeypatch.setattr(bisim, "bisim_get_stats", lambda ctx: stats)
    monkeypatch.setattr(bisim, "bisim_autotune", fake_autotune)
    monkeypatch.setattr(bisim, "bisim_retune", lambda ctx, stream=None, **kw: calls["retune"].append(kw))
    monkeypatch.setattr(tuning, "_device_name", lambda: "GPU A")
    cache = tuning.TuneCache(str(tmp_path / "t.json"))
    got, hit = tuning.autotune_cached(object(), cache)
    assert (got, hit, calls["autotune"], calls["retune"]) == (chosen, False, 1, [])
    fresh = tuning.TuneCache(str(tmp_path / "t.json"))
    got, hit = tuning.autotune_cached(object(), fresh)
    assert (got, hit, calls["autotune"]) == (chosen, True, 1)
    assert calls["retune"] == [chosen]
    # another shape is tuned again
    stats["n_edges"] = 50_000_000
    _, hit = tuning.autotune_cached(object(), fresh)
    assert not hit and calls["autotune"] == 2


def test_retune_rejects_other_fields():
    with pytest.raises(ValueError):
        bisim.bisim_retune(object(), flags=1)
