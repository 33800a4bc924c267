"""Host-side pieces of the benchmark, without a GPU: the clock summary parsed
from nvidia-smi lines, the profiled DRAM traffic that holds only while the
trace kernel's sources are unchanged, and the precision report's masks and
error measures.
"""
import os
import re

import numpy as np

import bench
from paper_1012_2865_gb300 import synth


def test_clock_summary():
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2002, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
               "1980, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line",
               "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2002.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_profiled_traffic_holds_only_for_the_profiled_sources(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "trace_kernel_fp32_mixed_stromgren128.md")
    text = open(path).read()
    recorded = re.search(r"kernel_source_sha256: `([0-9a-f]{64})`", text).group(1)
    traffic = float(re.search(r"dram_bytes_per_launch: `?([0-9.eE+]+)", text).group(1))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: recorded)
    assert bench._profiled_traffic("fp32_mixed", "stromgren128") == traffic
    assert bench._profiled_traffic("fp32_mixed", "no_such_workload") is None
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "0" * 64)
    assert bench._profiled_traffic("fp32_mixed", "stromgren128") is None


def test_precision_report():
    g = synth.stromgren_snapshot(32)
    n = g["n_H"].size
    rng = np.random.default_rng(0)
    kph = rng.uniform(1e-14, 1e-12, n)
    kph[:10] = 0.0  # cells receiving nothing are not compared
    x = rng.uniform(1e-6, 1.0, n)
    emitted = 1e40
    ref = (kph, x, emitted)
    final = {"fp64": {"kph": kph.copy(), "x_HI": x.copy()},
             "fp32_mixed": {"kph": kph * (1 + 3e-6), "x_HI": x * (1 - 1e-6)}}
    rep = bench.precision_error(g, ref, final)
    assert rep["cells_compared_kph"] == n - 10
    assert rep["fp64"]["kph_max_rel"] == 0.0 and rep["fp64"]["x_HI_max_rel"] == 0.0
    np.testing.assert_allclose(rep["fp32_mixed"]["kph_max_rel"], 3e-6, rtol=1e-6)
    np.testing.assert_allclose(rep["fp32_mixed"]["x_HI_median_rel"], 1e-6, rtol=1e-6)


def test_threaded_oracle_step_equals_the_oracle_step():
    """The CPU baseline's threaded step (root packages shared by host threads,
    thread-private k_ph summed, the update on cell ranges) gives the oracle's
    step: the same segments and emitted photons, k_ph to summation order and
    the same x_HI."""
    import numpy as np
    from paper_1012_2865_gb300 import synth
    g = synth.stromgren_snapshot(32)
    s1, k1, x1, e1 = bench.oracle_step(g, g["x_HI"], g["x_HII"])
    s4, k4, x4, e4 = bench.oracle_step_threads(g, g["x_HI"], g["x_HII"], 4)
    assert s1 == s4
    assert abs(e1 - e4) <= 1e-12 * e1
    m = k1 > 0
    assert np.array_equal(k4 > 0, m)
    assert np.max(np.abs(k4[m] - k1[m]) / k1[m]) < 1e-12
    assert np.allclose(x4, x1, rtol=1e-12, atol=1e-15)
