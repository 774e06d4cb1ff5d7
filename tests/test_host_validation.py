"""Host-side validation of the C ABI, without a GPU: aeth_create,
aeth_add_block, aeth_link_blocks and aeth_plan run on the host (no CUDA
call before aeth_finalize), so their argument checks, their rejection of
combinations that are not built, the call order and the arena sizing are
tested here through the real library."""
import math

import pytest

from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import build as B

ARG, STATE, UNSUP = -1, -7, -8


@pytest.fixture(scope="module", autouse=True)
def _library():
    B.build()
    A.load_library()


def _create_code(cfg):
    try:
        ctx = A.aeth_create(cfg)
    except A.AethError as e:
        return e.code
    A.aeth_destroy(ctx)
    return 0


def _cfg(**kw):
    """make_config arguments, then raw field overrides given as field=value
    under the key 'raw'."""
    raw = kw.pop("raw", {})
    cfg = A.make_config(**kw)
    for k, v in raw.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("kw", [
    dict(raw=dict(eos=7)),
    dict(gamma=1.0),
    dict(gamma=float("nan")),
    dict(iso=True, cs=0.0),
    dict(iso=True, cs=float("inf")),
    dict(iso=True, cs=float("nan")),
    dict(raw=dict(recon=4)),
    dict(raw=dict(riemann=4)),
    dict(raw=dict(integrator=4)),
    dict(raw=dict(precision=4)),
    dict(cfl=0.0),
    dict(cfl=1.5),
    dict(cfl=float("nan")),
    dict(raw=dict(path=2)),
    dict(raw=dict(drag_precision=3)),
    dict(raw=dict(mlp_engine=2)),
    dict(raw=dict(n_dust=33)),
    dict(raw=dict(n_dust=2)),                              # no stopping times given
    dict(mhd=False, integrator=A.IMEX2P, t_stop=[0.1, 0.0]),
    dict(mhd=False, integrator=A.IMEX2P, t_stop=[0.1, -1.0]),
    dict(raw=dict(drag_law=2)),
])
def test_create_rejects_invalid_values(kw):
    assert _create_code(_cfg(**kw)) == ARG


@pytest.mark.parametrize("kw", [
    dict(t_stop=[0.1], integrator=A.IMEX2P),               # dust under MHD gas
    dict(t_stop=[0.1], mhd=False),                         # dust without IMEX2P
    dict(mhd=False, integrator=A.IMEX2P),                  # IMEX2P without dust
    dict(t_stop=[0.1], mhd=False, integrator=A.IMEX2P, drag_law=A.DRAG_COEFF,
         precision=A.FP32, drag_precision=A.DRAG_SEL64),   # per-species choice needs t_k
    dict(dual=True, iso=True),
    dict(dual=True, precision=A.FP32_SEL64),
    dict(dual=True, path=A.UNFUSED),
    dict(dual=True, precision=A.FP32_P64),
    dict(dual=True, riemann=A.MLP, precision=A.FP32),
    dict(dual=True, mhd=False, integrator=A.IMEX2P, t_stop=[0.1]),
    dict(iso=True, riemann=A.LHLLD),
    dict(riemann=A.MLP, precision=A.FP64),
    dict(riemann=A.MLP, precision=A.FP32, mhd=False, integrator=A.IMEX2P, t_stop=[0.1]),
    dict(riemann=A.MLP, precision=A.FP32, iso=True),
])
def test_create_rejects_combinations_not_built(kw):
    assert _create_code(_cfg(**kw)) == UNSUP


@pytest.mark.parametrize("kw", [
    dict(),
    dict(precision=A.FP32, recon=A.PPM5, integrator=A.RK3, riemann=A.LHLLD),
    dict(precision=A.FP32_P64, riemann=A.HLLE, integrator=A.RK2, path=A.UNFUSED),
    dict(iso=True, cs=0.5, mhd=False, recon=A.PPM),
    dict(dual=True, precision=A.FP32),
    dict(mhd=False, integrator=A.IMEX2P, t_stop=[1e-4, 1e-2, 1.0], precision=A.FP32,
         drag_precision=A.FP32),
    dict(riemann=A.MLP, precision=A.FP32, mlp_engine=A.MMA_SYNC),
    dict(precision=A.FP32_SEL64, p64_ratio=8.0),
    dict(mhd=False, integrator=A.IMEX2P, t_stop=[1e-4, 1.0], precision=A.FP32,
         drag_precision=A.DRAG_SEL64, drag_ratio=2.0),
    dict(t_stop=[1.0, 3.0], mhd=False, integrator=A.IMEX2P, iso=True, drag_law=A.DRAG_COEFF),
])
def test_create_accepts_every_built_family(kw):
    assert _create_code(_cfg(**kw)) == 0


def _with_ctx(cfg, fn):
    ctx = A.aeth_create(cfg)
    try:
        return fn(ctx)
    finally:
        A.aeth_destroy(ctx)


def _add_code(cfg, desc):
    def go(ctx):
        try:
            A.aeth_add_block(ctx, desc)
        except A.AethError as e:
            return e.code
        return 0
    return _with_ctx(cfg, go)


SPH_LO, SPH_HI = (1.0, math.pi / 4, 0.0), (2.0, 3 * math.pi / 4, math.pi / 2)


@pytest.mark.parametrize("desc,cfg,code", [
    (A.make_block((0, 8, 8)), dict(), ARG),
    (A.make_block((8, 8, 8), lo=(1.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)), dict(), ARG),
    (A.make_block((8, 8, 8), coord=2), dict(), ARG),
    (A.make_block((8, 8, 8), bc=(A.PERIODIC, 5, A.PERIODIC)), dict(), ARG),
    (A.make_block((2048, 1024, 1025)), dict(), ARG),                  # more than 2^31 cells
    # a periodic axis shorter than the ghost width (PPM: 3) wraps onto itself
    (A.make_block((2, 8, 8)), dict(recon=A.PPM), ARG),
    (A.make_block((1, 8, 8)), dict(recon=A.PPM), 0),                  # n = 1: uniform axis
    (A.make_block((8, 8, 8), lo=SPH_LO, hi=SPH_HI, coord=A.SPH,
                  bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)), dict(integrator=A.RK3), UNSUP),
    (A.make_block((8, 8, 8), lo=SPH_LO, hi=SPH_HI, coord=A.SPH,
                  bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)),
     dict(mhd=False, integrator=A.IMEX2P, t_stop=[0.1]), UNSUP),
    # r including the ghost layers must stay positive, theta off the axis
    (A.make_block((4, 8, 8), lo=(0.1, 1.0, 0.0), hi=(0.5, 2.0, 1.0), coord=A.SPH,
                  bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)), dict(), ARG),
    (A.make_block((8, 8, 8), lo=(1.0, 0.05, 0.0), hi=(2.0, 1.0, 1.0), coord=A.SPH,
                  bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)), dict(), ARG),
    (A.make_block((8, 8, 8), lo=SPH_LO, hi=SPH_HI, coord=A.SPH,
                  bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)), dict(), 0),
])
def test_add_block_validation(desc, cfg, code):
    assert _add_code(A.make_config(**cfg), desc) == code


def test_link_validation():
    d = [A.make_block((8, 8, 8)), A.make_block((8, 6, 8), hi=(1.0, 0.75, 1.0))]

    def go(ctx):
        for b in d:
            A.aeth_add_block(ctx, b)
        with pytest.raises(A.AethError) as e:
            A.aeth_link_blocks(ctx, 0, 0, 1)          # ny differs across the x face
        assert e.value.code == ARG
        A.aeth_link_blocks(ctx, 0, 1, 1)              # along y: nx, nz agree
        for args in ((0, 1, 1), (0, 3, 1), (0, 0, 2), (-1, 0, 1)):
            with pytest.raises(A.AethError) as e:     # linked twice, bad axis, bad index
                A.aeth_link_blocks(ctx, *args)
            assert e.value.code == ARG
    _with_ctx(A.make_config(), go)
    # a different cell width, a transverse offset, too few cells along the
    # link axis for the ghost width, a spherical block
    for other, code in ((A.make_block((8, 8, 8), hi=(2.0, 1.0, 1.0)), ARG),
                        (A.make_block((8, 8, 8), lo=(0.0, 0.5, 0.0), hi=(1.0, 1.5, 1.0)), ARG),
                        (A.make_block((1, 8, 8), hi=(0.125, 1.0, 1.0)), ARG),
                        (A.make_block((8, 8, 8), lo=SPH_LO, hi=SPH_HI, coord=A.SPH,
                                      bc=(A.OUTFLOW, A.OUTFLOW, A.PERIODIC)), UNSUP)):
        def go2(ctx, other=other, code=code):
            A.aeth_add_block(ctx, d[0])
            A.aeth_add_block(ctx, other)
            with pytest.raises(A.AethError) as e:
                A.aeth_link_blocks(ctx, 0, 0, 1)
            assert e.value.code == code
        _with_ctx(A.make_config(), go2)
    # the unfused path and dust runs have no linked blocks
    for cfg in (A.make_config(path=A.UNFUSED),
                A.make_config(mhd=False, integrator=A.IMEX2P, t_stop=[0.1])):
        def go3(ctx):
            A.aeth_add_block(ctx, d[0])
            with pytest.raises(A.AethError) as e:
                A.aeth_link_blocks(ctx, 0, 0, 0)
            assert e.value.code == UNSUP
        _with_ctx(cfg, go3)


def test_call_order():
    def go(ctx):
        with pytest.raises(A.AethError) as e:
            A.aeth_plan(ctx)                          # no blocks yet
        assert e.value.code == STATE
        A.aeth_add_block(ctx, A.make_block((8, 8, 8)))
        A.aeth_plan(ctx)
        for call in (lambda: A.aeth_add_block(ctx, A.make_block((8, 8, 8))),
                     lambda: A.aeth_link_blocks(ctx, 0, 0, 0)):
            with pytest.raises(A.AethError) as e:
                call()
            assert e.value.code == STATE
        assert "before plan" in A.aeth_last_error(ctx)
    _with_ctx(A.make_config(), go)


def _plan_bytes(cfg, blocks):
    def go(ctx):
        for b in blocks:
            A.aeth_add_block(ctx, b)
        return A.aeth_plan(ctx)
    return _with_ctx(cfg, go)


def test_plan_arena_accounts_for_every_array():
    n = (32, 24, 16)
    blk = [A.make_block(n)]
    cells = 32 * 24 * 16
    b64 = _plan_bytes(A.make_config(), blk)
    b32 = _plan_bytes(A.make_config(precision=A.FP32), blk)
    # two registers of 8 variables at least, in the working precision
    assert b64 >= 2 * 8 * cells * 8 and b32 >= 2 * 8 * cells * 4
    assert 1.6 < b64 / b32 < 2.1
    # each extra set of arrays adds at least its unpadded size
    hydro = dict(mhd=False, integrator=A.IMEX2P)
    base = _plan_bytes(A.make_config(mhd=False), blk)
    d3 = _plan_bytes(A.make_config(t_stop=[0.1] * 3, **hydro), blk)
    assert d3 - base >= (2 * 4 + 12) * 3 * cells * 8
    dual = _plan_bytes(A.make_config(dual=True), blk)
    assert dual - b64 >= 2 * cells * 8
    mlp = _plan_bytes(A.make_config(riemann=A.MLP, precision=A.FP32), blk)
    assert mlp - b32 >= 45 * cells * 4
    # more blocks, more arena; a plan is deterministic
    two = _plan_bytes(A.make_config(), blk + [A.make_block((16, 16, 16))])
    assert two > b64
    assert _plan_bytes(A.make_config(), blk) == b64


@pytest.mark.parametrize("name,cfg,n", [
    ("512^3 learned flux, FP32", dict(riemann=A.MLP, precision=A.FP32), (512, 512, 512)),
    ("512x512x256 linear wave, FP64", dict(riemann=A.HLLE, integrator=A.RK2), (512, 512, 256)),
    ("256^3 turbulence, dual energy, FP64", dict(dual=True), (256, 256, 256)),
])
def test_largest_workloads_fit_in_hbm(name, cfg, n):
    # the device arena of each workload stays well inside the GB300's HBM
    # (288 GB, of which about 280 GB are usable)
    need = _plan_bytes(A.make_config(**cfg), [A.make_block(n)])
    assert need < 200e9, (name, need / 1e9)
