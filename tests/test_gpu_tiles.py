"""Flux-tile shapes and their autotuner on the GPU.

The flux pass gives each face to exactly one thread whatever the tile
shape, so the 32 x 4 and 16 x 8 tiles, with any z-chunk, give the same
state bit for bit: on one ragged block and on uneven linked and unlinked
blocks.  The band tiles (whole rows of a block) run the same arithmetic in
a kernel the compiler arranges differently, and its multiply-add
contractions differ in a few per cent of the faces: their states agree
with the 2-D tiles' to a few FP32 ulps, and with the oracle at the FP32
bound on narrow, ragged and 64-wide blocks.  The autotuner picks a built shape, and Solver.tune_tiles
stores it in its JSON cache and takes it from there the second time."""
import numpy as np
import pytest

from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(states, tile, steps=2, cfg=None, links=()):
    import torch
    cfg = cfg or A.make_config(gamma=states[0].gamma, precision=A.FP32)
    blocks = [A.make_block(s.block.n, s.block.lo, s.block.hi, s.block.coord, s.block.bc)
              for s in states]
    sv = A.Solver(cfg, blocks, stream=torch.cuda.current_stream(), links=links)
    try:
        if tile is not None:
            A.aeth_set_flux_tile(sv.ctx, *tile)
            assert A.aeth_get_flux_tile(sv.ctx) == tuple(tile)
        for q, s in enumerate(states):
            sv.set_state(q, s.cons, s.b1, s.b2, s.b3)
        for _ in range(steps):
            sv.step(2e-3)
        return [sv.get_state(q) for q in range(len(states))]
    finally:
        sv.close()


def _same(a, b):
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def _close(a, b, ulps=8):
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            d = float(np.max(np.abs(u.astype(np.float64) - v)))
            assert d <= ulps * 2.0 ** -23 * float(np.max(np.abs(u))), d


@pytest.mark.parametrize("recon", [A.PLM, A.PPM])
def test_tile_shapes_give_identical_states(recon):
    st = I.smooth_random_mhd(I.Block((40, 20, 12)), 5, v_rms=0.5, b_rms=0.5)
    cfg = A.make_config(gamma=st.gamma, precision=A.FP32, recon=recon)
    ref = _run([st], (32, 16), cfg=cfg)
    for tile in ((16, 16), (16, 3), (32, 5), (16, 64)):
        _same(ref, _run([st], tile, cfg=cfg))
    band = _run([st], (0, 16), cfg=cfg)
    _close(ref, band)
    _same(band, _run([st], (0, 3), cfg=cfg))   # band tiles: any z-chunk


def test_tile_shapes_identical_on_uneven_blocks():
    sts = [I.smooth_random_mhd(I.Block(n), 60 + q, v_rms=0.4, b_rms=0.5)
           for q, n in enumerate(((17, 9, 12), (24, 16, 8), (33, 20, 10)))]
    ref = _run(sts, (32, 16))
    _same(ref, _run(sts, (16, 8)))
    _close(ref, _run(sts, (0, 8)))


@pytest.mark.parametrize("recon", ["plm", "ppm"])
def test_band_tiles_parity_on_narrow_ragged_and_widest_blocks(recon):
    # widths 1 (three flux columns), 14 (16 columns: the band rows fill the
    # 256 threads exactly), 17 (ragged: 13 rows and 22 idle threads) and 64
    # (the widest band, three rows); each block is its own periodic box, so
    # the oracle advances each alone with the same dt sequence
    from tests.gpu_helpers import RECON, compare, oracle_run
    sts = [I.smooth_random_mhd(I.Block(n), 70 + q, v_rms=0.4, b_rms=0.5)
           for q, n in enumerate(((1, 12, 6), (14, 9, 7), (17, 11, 5), (64, 7, 4)))]
    dts = [4e-4] * 3
    cfg = A.make_config(gamma=sts[0].gamma, precision=A.FP32, recon=RECON[recon][1])
    import torch
    blocks = [A.make_block(s.block.n, s.block.lo, s.block.hi, s.block.coord, s.block.bc)
              for s in sts]
    sv = A.Solver(cfg, blocks, stream=torch.cuda.current_stream())
    try:
        A.aeth_set_flux_tile(sv.ctx, 0, 4)
        for q, s in enumerate(sts):
            sv.set_state(q, s.cons, s.b1, s.b2, s.b3)
        for dt in dts:
            sv.step(dt)
        band = [sv.get_state(q) for q in range(len(sts))]
    finally:
        sv.close()
    for q, s in enumerate(sts):
        ref, _ = oracle_run(s, recon, "vl2", dts=dts)
        e = compare(band[q], ref)
        assert max(e) < 1e-5, (q, e)


def test_tile_shape_rejections():
    import torch
    sv = A.Solver(A.make_config(precision=A.FP32), [A.make_block((8, 8, 8))],
                  stream=torch.cuda.current_stream())
    try:
        for bad in ((24, 16), (16, 0), (32, 5000)):
            with pytest.raises(A.AethError) as e:
                A.aeth_set_flux_tile(sv.ctx, *bad)
            assert e.value.code == -1
    finally:
        sv.close()
    # band tiles take blocks at most 64 cells wide
    sv = A.Solver(A.make_config(precision=A.FP32), [A.make_block((65, 4, 4))],
                  stream=torch.cuda.current_stream())
    try:
        with pytest.raises(A.AethError) as e:
            A.aeth_set_flux_tile(sv.ctx, 0, 8)
        assert e.value.code == -8
    finally:
        sv.close()
    sv = A.Solver(A.make_config(precision=A.FP64), [A.make_block((8, 8, 8))],
                  stream=torch.cuda.current_stream())
    try:
        with pytest.raises(A.AethError) as e:
            A.aeth_set_flux_tile(sv.ctx, 16, 16)
        assert e.value.code == -8
        A.aeth_set_flux_tile(sv.ctx, 32, 16)       # the 32-wide tile is always built
    finally:
        sv.close()


def test_autotuner_and_its_cache(tmp_path):
    import torch
    st = I.smooth_random_mhd(I.Block((48, 40, 32)), 8, v_rms=0.5, b_rms=0.5)
    cfg = A.make_config(gamma=st.gamma, precision=A.FP32)
    cache = str(tmp_path / "tiles.json")
    got = []
    for _ in range(2):
        sv = A.Solver(cfg, [A.make_block((48, 40, 32))], stream=torch.cuda.current_stream())
        try:
            sv.set_state(0, st.cons, st.b1, st.b2, st.b3)
            got.append(sv.tune_tiles(cache=cache, device="test"))
            assert A.aeth_get_flux_tile(sv.ctx) == got[-1][:2]
        finally:
            sv.close()
    assert got[0][2] == "tuned" and got[1][2] == "cache"
    assert got[0][:2] == got[1][:2]
    assert got[0][0] in (0, 16, 32) and got[0][1] in (8, 16, 32, 64)
