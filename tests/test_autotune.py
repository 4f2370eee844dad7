"""Host logic of the tile-size autotuner (no GPU)."""
from paper_2411_17660_b300 import autotune as A
from paper_2411_17660_b300.render import Intrinsics


def test_choose_picks_fastest_and_breaks_ties_in_order():
    times = {8: 3.0, 16: 1.5, 32: 2.0}
    r = A.choose(lambda t: times[t])
    assert r["tile"] == 16 and r["ms"] == times
    r = A.choose(lambda t: 1.0)
    assert r["tile"] == 8


def test_signature_distinguishes_views_and_sizes():
    c1 = [Intrinsics(480, 640, 500, 500, 320, 240)]
    c2 = [Intrinsics(240, 320, 250, 250, 160, 120)]
    assert A.signature("B300", 10, 3, c1) != A.signature("B300", 10, 3, c2)
    assert A.signature("B300", 10, 3, c1) != A.signature("B300", 11, 3, c1)
    assert A.signature("B300", 10, 3, c1) == A.signature("B300", 10, 3, list(c1))


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tiles.json")
    c = A.TileCache(path)
    assert c.get("k") is None
    c.put("k", {"tile": 32, "ms": {"8": 1.0}})
    again = A.TileCache(path)
    assert again.get("k")["tile"] == 32
