"""Host logic of the tile-size autotuner (no GPU)."""
from paper_2411_17660_b300 import autotune as A
from paper_2411_17660_b300.render import Intrinsics


def test_choose_picks_fastest_and_breaks_ties_in_order():
    times = {"8/tile": 3.0, "8/radix": 2.5, "16/tile": 1.5, "16/radix": 1.7, "32/tile": 2.0, "32/radix": 1.6}
    r = A.choose(lambda c: times[c])
    assert r["best"] == "16/tile" and r["ms"] == times
    r = A.choose(lambda c: 1.0)
    assert r["best"] == A.CANDIDATES[0]


def test_candidates_cover_every_tile_size_and_binning():
    assert {A.parse(c) for c in A.CANDIDATES} == {(t, b) for t in A.TILES for b in A.BINNINGS}
    assert A.parse("32/radix") == (32, "radix")


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
