"""Host-side logic without a GPU: the mesh-block decomposition helper, the
bench's block splitting and its option checks."""
import numpy as np
import pytest

import bench
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I


def test_decompose_counts_links_and_extents():
    n = (24, 20, 14)
    splits = ([9, 15], [8, 5, 7], [6, 8])
    descs, links, origin = A.decompose(n, splits, (0.0, -1.0, 0.0), (2.4, 1.0, 1.4),
                                       (A.PERIODIC, A.OUTFLOW, A.PERIODIC))
    assert len(descs) == 12
    # periodic x and z wrap (2 links per row / column), outflow y does not
    assert len(links) == 12 + 8 + 12
    assert len(set((lo, ax) for lo, ax, _ in links)) == len(links)   # each high side once
    assert len(set((hi, ax) for _, ax, hi in links)) == len(links)   # each low side once
    for q, (d, o) in enumerate(zip(descs, origin)):
        # extents follow the cell offsets with the domain's uniform spacing
        assert d.x1min == pytest.approx(0.1 * o[0])
        assert d.x1max == pytest.approx(0.1 * (o[0] + d.nx))
        assert d.x2min == pytest.approx(-1.0 + 0.1 * o[1])
        assert d.x3max == pytest.approx(0.1 * (o[2] + d.nz))
    for lo, ax, hi in links:
        a, b = origin[lo], origin[hi]
        na = (descs[lo].nx, descs[lo].ny, descs[lo].nz)
        assert b[ax] == (a[ax] + na[ax]) % n[ax]
        for e in range(3):
            if e != ax:
                assert a[e] == b[e]


def test_decompose_single_block_links_itself_on_periodic_axes():
    descs, links, origin = A.decompose((8, 8, 8), ([8], [8], [8]),
                                       bc=(A.PERIODIC, A.OUTFLOW, A.PERIODIC))
    assert links == [(0, 0, 0), (0, 2, 0)]
    assert origin == [(0, 0, 0)]


def test_bench_split_into_blocks_reassembles_the_state():
    st = I.smooth_random_mhd(I.Block((16, 8, 8)), 3, v_rms=0.5, b_rms=0.5)
    parts, descs, links = bench.split_into_blocks(A, st, 8)
    assert len(parts) == 2 and len(links) == 6
    whole = np.concatenate([parts[0].cons, parts[1].cons], axis=3)
    np.testing.assert_array_equal(whole, st.cons)
    # the shared x face appears in both blocks with the same values
    np.testing.assert_array_equal(parts[0].b1[..., -1], parts[1].b1[..., 0])
    with pytest.raises(SystemExit):
        bench.split_into_blocks(A, st, 6)


@pytest.mark.parametrize("argv", [["--dual", "--prec", "fp32_p64"], ["--iso", "--workload", "wave512"],
                                  ["--block-size", "64", "--workload", "dust128"],
                                  ["--dual", "--iso"]])
def test_bench_rejects_option_combinations(argv):
    with pytest.raises(SystemExit):
        bench.parse(argv)


def test_bench_workload_names():
    assert bench.workload_config(bench.parse(["--dual"]))["workload"].endswith("_dual_energy")
    a = bench.parse(["--workload", "wave512", "--block-size", "128"])
    cfg = bench.workload_config(a)
    assert cfg["workload"] == "linear_wave_512x512x256_mhd_blocks128"
    assert cfg["blocks"].startswith("32 linked blocks")
    assert bench.parse(["--workload", "wave512"]).prec == "fp64"


def test_issue_roofline_and_alu_peaks_helpers():
    # issue roofline: instructions per launch over the launch time, against
    # 4 slots per SM per cycle; absent figures give None
    r = bench.issue_roofline("fused_fp32_plm", 1.5, 2000.0, 100)
    if r is not None:   # present while the committed figures match the kernel source
        assert r["peak"] == pytest.approx(4 * 100 * 2000e6 / 1e12)
        assert r["achieved"] == pytest.approx(r["warp_inst_per_launch"] / 1.5e-3 / 1e12)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.issue_roofline("no_such_key", 1.5, 2000.0) is None
    assert bench.issue_roofline("fused_fp32_plm", 0.0, 2000.0) is None

    class FakeA:
        FP32, FP64 = 1, 0

        @staticmethod
        def aeth_probe_fma(prec):
            return 8e13 if prec == 1 else 1.25e12

    p = bench.alu_peaks(FakeA)
    assert p["fp32_tflops"] == pytest.approx(80.0) and p["fp64_tflops"] == pytest.approx(1.25)

    class Broken(FakeA):
        @staticmethod
        def aeth_probe_fma(prec):
            raise RuntimeError("no device")

    assert "error" in bench.alu_peaks(Broken)


def test_committed_traffic_figures_match_the_kernel_source():
    """The committed ncu figures are keyed to the flux kernel's code; the
    default workload's entry must match the current source."""
    assert bench.ncu_traffic("fused_fp32_plm") is not None
    assert bench.ncu_figure("fused_fp32_plm", "warp_inst_per_launch") is not None


def test_reference_sample_size_keeps_the_reference_arm_within_minutes():
    # fits: the probe size stays
    assert bench.reference_sample_size(0.3, 64, 20) == 64
    # too long: the cell count shrinks with the budget (n^3 scaling), to a
    # multiple of 8, never below 16
    n = bench.reference_sample_size(0.3, 64, 1000)
    assert n % 8 == 0 and 16 <= n < 64
    assert 1000 * 0.3 * (n / 64) ** 3 <= 150.0
    assert bench.reference_sample_size(0.3, 64, 10 ** 7) == 16


@pytest.mark.parametrize("argv", [["--steps", "0"], ["--warmup", "-1"]])
def test_bench_rejects_empty_timing(argv):
    with pytest.raises(SystemExit):
        bench.parse(argv)


def test_single_thread_oracle_rate_runs_in_a_child_process():
    r = bench.single_thread_rate(bench.parse(["--workload", "wave32"]), 8, seconds=0.2)
    assert r["value"] > 0 and r["steps"] >= 1 and "fast wave 8^3" in r["what"]


def test_packed_state_layout_is_block_after_block():
    """pack_states: each block's cons, then its three face fields (MHD), then
    its dust species, block after block (the layout of the packed transfers)."""
    rng = np.random.default_rng(3)
    blocks = []
    for n in ((3, 2, 2), (2, 4, 1)):
        nx, ny, nz = n
        blocks.append((rng.random((5, nz, ny, nx)), rng.random((nz, ny, nx + 1)),
                       rng.random((nz, ny + 1, nx)), rng.random((nz + 1, ny, nx))))
    dust = [rng.random((2, 4) + b[0].shape[1:]) for b in blocks]
    p = A.pack_states(blocks, mhd=True, dust=dust)
    o = 0
    for b, d in zip(blocks, dust):
        for arr in list(b) + [d]:
            assert np.array_equal(p[o:o + arr.size], arr.ravel())
            o += arr.size
    assert o == p.size
    h = A.pack_states([(b[0],) for b in blocks], mhd=False)
    assert h.size == sum(b[0].size for b in blocks)
