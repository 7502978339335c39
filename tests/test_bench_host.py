"""Host-side pieces of the benchmark (no GPU): the clock record that decides
whether a timed run saw throttling, and the kernel-source stamp that gates
the reported DRAM traffic."""
import bench


def test_clock_record_median_and_throttle_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    r = bench.parse_clocks(lines)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clocks(["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active\n"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clocks([])["sm_mhz"] is None


def test_kernel_source_stamp_ignores_comments_and_spacing():
    """The stamp hashes code only: it is stable across calls and is a 16-digit
    hex string (a changed comment does not void the traffic record)."""
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash() and len(h) == 16 and int(h, 16) >= 0
