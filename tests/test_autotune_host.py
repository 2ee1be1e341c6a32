"""Host logic of the autotuner: the partition prior orders candidates, the
cache round-trips, lookups fall back to the default."""
from paper_1508_02977_gb300 import autotune, partition


def test_prior_prefers_large_area_to_perimeter():
    cands = [((64, 16), 0, 2), ((32, 32), 0, 2), ((48, 48), 0, 2), ((32, 32), 2, 2)]
    order = autotune.prior_order(cands, 3840, 2160)
    assert order[0] == ((48, 48), 0, 2)
    # equal tiles: the one without overlap first
    assert order.index(((32, 32), 0, 2)) < order.index(((32, 32), 2, 2))
    # 64x16 has a smaller area/perimeter ratio than 32x32 (same area)
    assert partition.part_ratio(64, 16, 1, 1) < partition.part_ratio(32, 32, 1, 1)
    assert order.index(((32, 32), 0, 2)) < order.index(((64, 16), 0, 2))


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.lookup(640, 480, 1, "GB300", path) == autotune.FALLBACK
    d = autotune.load_cache(path)
    d[autotune._key(640, 480, 1, "GB300")] = {"tile": [32, 32], "overlap": 0, "sweeps": 2, "ms": 1.0}
    autotune.save_cache(d, path)
    assert autotune.lookup(700, 500, 1, "GB300", path) == {"tile": (32, 32), "overlap": 0, "sweeps": 2, "omega": 1.0}
    d[autotune._key(640, 480, 1, "GB300")]["omega"] = 1.6
    autotune.save_cache(d, path)
    assert autotune.lookup(700, 500, 1, "GB300", path)["omega"] == 1.6
    # another size class or precision is not matched
    assert autotune.lookup(3840, 2160, 1, "GB300", path) == autotune.FALLBACK
    assert autotune.lookup(640, 480, 0, "GB300", path) == autotune.FALLBACK
