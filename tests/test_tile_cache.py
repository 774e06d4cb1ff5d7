"""Host logic of the flux-tile cache (no GPU): the key follows the
configuration, the block-size multiset and the device, and the JSON file
round-trips and survives a broken file."""
import json

from paper_2608_14048_gb300 import aether as A


def test_key_depends_on_what_changes_the_flux_pass():
    cfg = A.make_config(precision=A.FP32)
    b = [A.make_block((16, 24, 32)), A.make_block((64, 16, 16))]
    k0, body = A.tile_cache_key(cfg, b, "GB300")
    assert A.tile_cache_key(cfg, list(reversed(b)), "GB300")[0] == k0   # a multiset
    assert A.tile_cache_key(cfg, b + b[:1], "GB300")[0] != k0
    assert A.tile_cache_key(cfg, b, "other GPU")[0] != k0
    cfg2 = A.make_config(precision=A.FP32, recon=A.PPM)
    assert A.tile_cache_key(cfg2, b, "GB300")[0] != k0
    assert [list(x) for x in body["blocks"]] == [["16x24x32:0", 1], ["64x16x16:0", 1]]


def test_cache_file_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tiles.json")
    assert A.load_tile_cache(p) == {}
    A.store_tile_cache(p, "a", {"flux_tx": 16, "kchunk": 32})
    A.store_tile_cache(p, "b", {"flux_tx": 32, "kchunk": 8})
    d = A.load_tile_cache(p)
    assert d == {"a": {"flux_tx": 16, "kchunk": 32}, "b": {"flux_tx": 32, "kchunk": 8}}
    open(p, "w").write("{broken")
    assert A.load_tile_cache(p) == {}
    json.dump([1, 2], open(p, "w"))
    assert A.load_tile_cache(p) == {}
