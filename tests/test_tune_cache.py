"""The batched path's cache of tuned configurations (host logic, no GPU): the
key groups batches of the same GPU, dtype, path, request and shape buckets;
the JSON file round-trips, keeps other keys, and treats a damaged file as a
miss."""
import json

import paper_2005_03246_gb300 as fk

CC = (10, 3)
SHAPES = [(1000, 2), (5000, 3), (20000, 2)]


def test_key_is_stable_and_order_free():
    a = fk.tune_key(CC, 0, 0, 3, SHAPES)
    assert a == fk.tune_key(CC, 0, 0, 3, list(reversed(SHAPES)))
    assert a.startswith("sm103|") and "d2:2,d3:1" in a and "sets3" in a


def test_key_buckets_sizes_but_separates_what_matters():
    a = fk.tune_key(CC, 0, 0, 3, SHAPES)
    # a few percent more points stay in the same power-of-two buckets
    assert a == fk.tune_key(CC, 0, 0, 3, [(1050, 2), (5100, 3), (20500, 2)])
    assert a != fk.tune_key(CC, 0, 0, 3, [(n * 8, d) for n, d in SHAPES])      # 8x the points
    assert a != fk.tune_key(CC, 0, 0, 3, [(1000, 2), (5000, 2), (20000, 2)])  # another dimension mix
    assert a != fk.tune_key(CC, 1, 0, 3, SHAPES)                              # FP64 data
    assert a != fk.tune_key(CC, 0, 1, 3, SHAPES)                              # FP64 path
    assert a != fk.tune_key(CC, 0, 0, 1, SHAPES)                              # counts only
    assert a != fk.tune_key((10, 0), 0, 0, 3, SHAPES)                         # another GPU


def test_round_trip_keeps_other_keys(tmp_path):
    path = str(tmp_path / "tune.json")
    assert fk.tune_cache_get(path, "k1") is None
    cfg1 = {"streams": 8, "coarsen": 1, "kernel_tile": 2048, "count_tile": 1024}
    fk.tune_cache_put(path, "k1", cfg1, 12.5)
    fk.tune_cache_put(path, "k2", dict(cfg1, streams=4), 9.0)
    assert fk.tune_cache_get(path, "k1") == {"config": cfg1, "ms": 12.5}
    assert fk.tune_cache_get(path, "k2")["config"]["streams"] == 4
    assert sorted(json.load(open(path))) == ["k1", "k2"]
    assert not list(tmp_path.glob("*.tmp*"))


def test_damaged_file_is_a_miss_and_is_replaced(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert fk.tune_cache_get(str(path), "k") is None
    fk.tune_cache_put(str(path), "k", {"streams": 2}, 1.0)
    assert fk.tune_cache_get(str(path), "k")["config"] == {"streams": 2}
    path.write_text(json.dumps({"k": "garbage", "j": {"config": 3}}))
    assert fk.tune_cache_get(str(path), "k") is None and fk.tune_cache_get(str(path), "j") is None
    path.write_text("[1, 2]")
    assert fk.tune_cache_get(str(path), "k") is None


class _FakeLib:
    """Stands in for the C library so that Batched's tuning logic runs on the
    CPU: the tuner "chooses" a fixed configuration and counts its calls."""

    def __init__(self):
        self.tuned = 0
        self.calls = 0

    def fk_batched_config_default(self, cfg):
        c = cfg._obj
        c.streams, c.coarsen, c.kernel_tile, c.count_tile = 4, 0, 0, 0

    def fk_batched_autotune_workspace(self, *a):
        return 256

    def fk_batched_autotune(self, *a):
        self.tuned += 1
        cfg, ms = a[-2]._obj, a[-1]._obj
        cfg.streams, cfg.coarsen, cfg.kernel_tile, cfg.count_tile = 8, 1, 1, 2
        ms.value = 3.25
        return 0

    def fk_batched_workspace_ex(self, *a):
        return 256

    def fk_batched_ex(self, *a):
        self.calls += 1
        return 0


def test_batched_uses_the_cache(tmp_path, monkeypatch):
    import torch
    fake = _FakeLib()
    monkeypatch.setattr(fk._lib, "load", lambda: fake)
    monkeypatch.setattr(fk, "_prep_points", lambda x, d=None: x.contiguous())
    monkeypatch.setattr(fk, "_stream_ptr", lambda dev: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "get_device_capability", lambda *a, **k: (10, 3))
    xs = [torch.rand(300, 2), torch.rand(40, 3)]
    path = str(tmp_path / "tune.json")
    b1 = fk.Batched(xs, graph=False, config="tune", tune_cache=path)
    assert fake.tuned == 1 and not b1.tune_cached
    assert b1.config == {"streams": 8, "coarsen": 1, "kernel_tile": 1, "count_tile": 2} and b1.tune_ms == 3.25
    b2 = fk.Batched(xs, graph=False, config="tune", tune_cache=path)
    assert fake.tuned == 1 and b2.tune_cached and b2.config == b1.config and b2.tune_ms == 3.25
    # another batch shape is another key: tuned again, stored beside the first
    b3 = fk.Batched([torch.rand(300, 2)], graph=False, config="tune", tune_cache=path)
    assert fake.tuned == 2 and not b3.tune_cached
    assert len(json.load(open(path))) == 2
    # without a cache file every tuned construction tunes
    fk.Batched(xs, graph=False, config="tune")
    assert fake.tuned == 3
