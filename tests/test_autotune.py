"""Host logic of the autotuner (no GPU): candidate list, cache, signature.
The timing itself runs in the library (gsr_autotune, tests/test_parity_gpu.py)."""
from paper_2411_17660_b300 import autotune as A
from paper_2411_17660_b300.render import Intrinsics


def test_candidates_cover_every_tile_binning_batch_and_block_height():
    want = {(t, b, k, r) for t in A.TILES for b in A.BINNINGS for k in A.BATCHES for r in A.FWD_ROWS
            if not (t == 32 and k == 64) and not (t == 8 and r == 16)}
    assert {A.parse(c) for c in A.CANDIDATES} == want and len(A.CANDIDATES) == len(want) == 16
    assert A.parse("32/radix/32/8") == (32, "radix", 32, 8)
    # the library's order: tile, then binning, then batch, then forward rows
    assert A.CANDIDATES[:3] == ("8/tile/32/8", "8/tile/64/8", "8/radix/32/8")
    assert A.CANDIDATES[4:6] == ("16/tile/32/16", "16/tile/32/8")


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
    c.put("k", {"tile": 32, "binning": "radix", "batch": 32, "fwd_rows": 8, "ms": {"8/tile/32/8": 1.0}})
    again = A.TileCache(path)
    assert again.get("k")["tile"] == 32
