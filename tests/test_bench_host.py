"""Host-side arithmetic of bench.py, without a GPU.

The roofline object must be the algorithmic work of the source-to-target step
(the nominal FFT-convolution count per target times the targets) over the
dense kernel's own duration against the measured peak, with the executed
tensor work beside it; the DRAM traffic must come from a committed ncu summary
only while the kernel source still has the sha256 the summary names; the FP32
peak must be the measured one; the clock sampler must report throttle reasons
it sees.
"""
import os
import tempfile

import pytest

import bench


def test_dense_roofline_is_nominal_work_over_kernel_time():
    steps = [{"ms_m2l": 1.2, "ms_m2l_kernel": 1.0, "m2l_parents": 30000},
             {"ms_m2l": 1.2, "ms_m2l_kernel": 1.0, "m2l_parents": 30000}]
    r = bench.roofline_of(steps, 4, 240000, None)
    nominal = bench.m2l_flops_per_target(4) * 240000
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(nominal / 1.0e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None
    # the executed dense work and the whole stage ride along under their own keys
    flop = 3 * 2 * 512 * 13824 * 30000
    assert r["executed"]["achieved"] == pytest.approx(flop / 1.0e-3 / 1e12)
    assert r["stage"]["achieved"] == pytest.approx(nominal / 1.2e-3 / 1e12)


def test_fft_roofline_against_measured_fp32_peak():
    steps = [{"ms_m2l": 8.0, "ms_m2l_kernel": 0.0, "m2l_parents": 0}]
    r = bench.roofline_of(steps, 4, 100000, None, {"fp32_tflops": 70.0})
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(bench.m2l_flops_per_target(4) * 100000 / 8.0e-3 / 1e12)
    committed = bench.alu_peaks().get("fp32_tflops")
    assert r["peak"] == pytest.approx(committed if committed else 70.0)
    assert "measured" in r["peak_basis"]


def test_p2p_roofline_counts_pairs():
    steps = [{"ms_p2p": 1.0, "p2p_pairs": 10 ** 9}]
    r = bench.p2p_roofline(steps, {"fp32_tflops": 80.0, "rsqrt_gops": 5000.0})
    assert r["achieved"] == pytest.approx(20 * 1e9 / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_nominal_fft_count_at_order_4():
    # P = 32: 5 P^3 log2(P^3) + 2 P^2 (P/2 + 1)
    assert bench.m2l_flops_per_target(4) == 5 * 32 ** 3 * 15 + 2 * 32 * 32 * 17


def test_traffic_only_for_the_profiled_source():
    src = os.path.join(bench.ROOT, "paper_1906_10734_gb300", "csrc", "m2l_tc.cu")
    t = bench.profile_traffic(src)
    if t is not None:
        assert t > 1e8      # a full-size launch moves hundreds of MB
        # per tile width where the summary has it, else the launch's figure
        assert bench.profile_traffic(src, 256) > 1e8
        assert bench.profile_traffic(src, 100) == t
    with tempfile.NamedTemporaryFile("w", suffix=".cu", delete=False) as f:
        f.write("// another kernel source\n")
    try:
        assert bench.profile_traffic(f.name) is None
    finally:
        os.unlink(f.name)


def test_clock_summary_reports_reasons():
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2010, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
    out = s.summary()
    assert out["sm_mhz"] == 2010 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(s.path)


def test_dense_work_per_parent_by_order():
    assert bench.dense_flop_per_parent(4) == 3 * 2 * 512 * 216 * 64
    # Ng = 6: 1728 rows padded to 14 blocks of 128, 216 nodes padded to 224 per slot
    assert bench.dense_flop_per_parent(6) == 3 * 2 * 1792 * 216 * 224
