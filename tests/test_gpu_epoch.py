"""Queue epochs and record layouts of the FP32-mixed trace.

Queue records of traces without a finite speed of light are 32 bytes and
carry the low 16 bits of their trace's epoch; before an epoch would repeat
them, the trace's set-up clears the queue.  Records of traces with a finite
speed of light carry the package's age and take 48 bytes; a grid that
switches between the two gets a queue of the other layout.

* A grid traced once with a large tree, then 65,534 times with a small one
  (which leaves the large tree's records in the upper slots), then with
  another large tree whose epoch has the same low 16 bits as the first,
  gives what a fresh grid gives for that tree.
* A grid traced without, with, and again without a finite speed of light
  gives the first result again.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# traces 2 .. 65535 of a fresh grid; the next one takes epoch 65537, whose low
# 16 bits (1) are those of trace 1
N_SMALL = (1 << 16) - 2


def _lit(k):
    return k > 1e-8 * k.max()


def test_epoch_wrap_leaves_no_stale_record():
    ctx = parity.ctx()
    a = synth.stromgren_snapshot(32, t_myr=500.0)
    a2 = synth.stromgren_snapshot(32, t_myr=120.0)
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    ref = native.Grid(ctx, a2, "fp32_mixed")
    want = ref.trace(**p)
    want_k = ref.rates()["kph"]
    ref.close()
    probe = native.Grid(ctx, a, "fp32_mixed")
    big = probe.trace(**p)
    probe.close()
    # a fixed capacity: one launch per trace, no retries (one epoch each)
    q = dict(p, queue_capacity=2 * max(big["queue_peak"], want["queue_peak"]) + (1 << 16))

    grid = native.Grid(ctx, a, "fp32_mixed")
    first = grid.trace(**q)
    # (how many children pass through the queue depends on scheduling: those
    # placed in a free lane of the splitting warp do not)
    assert first["status"] == 0 and first["passes"] == 1 and first["queue_pushed"] > 0
    np.testing.assert_array_equal(first["counts"], big["counts"])
    n = grid.ncell
    native.rt_set_state(grid.h, np.ones(n), np.zeros(n))  # neutral: packages stop within a few cells
    small = dict(q, checksums=False)
    for _ in range(N_SMALL):
        grid.trace(sync=False, **small)
    s = native.rt_get_budget(grid.h)
    assert s["status"] == 0
    assert 0 < s["queue_pushed"] < first["queue_pushed"] // 4  # the upper slots still hold trace 1's records
    native.rt_set_state(grid.h, a2["x_HI"], a2["x_HII"])
    got = grid.trace(**q)
    assert got["status"] == 0
    np.testing.assert_array_equal(got["counts"], want["counts"])
    np.testing.assert_array_equal(got["hashes"], want["hashes"])
    assert got["segments"] == want["segments"]
    k = grid.rates()["kph"]
    m = _lit(want_k)
    np.testing.assert_allclose(k[m], want_k[m], rtol=1e-5)
    assert abs(got["absorbed"] - want["absorbed"]) <= 1e-9 * want["emitted"]
    grid.close()


def test_switching_the_speed_of_light_keeps_results():
    ctx = parity.ctx()
    g = synth.stromgren_snapshot(32)
    dx = g["box_len_cm"] / 32
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    grid = native.Grid(ctx, g, "fp32_mixed")
    ref = grid.trace(**p)
    ref_k = grid.rates()["kph"]
    for _ in range(3):
        b = grid.trace(light_cm=2.5 * dx, **p)
        assert b["status"] == 0 and b["n_halted"] > 0
    got = grid.trace(**p)
    np.testing.assert_array_equal(got["counts"], ref["counts"])
    np.testing.assert_array_equal(got["hashes"], ref["hashes"])
    assert got["segments"] == ref["segments"] and got["n_resumed"] == 0
    k = grid.rates()["kph"]
    m = _lit(ref_k)
    np.testing.assert_allclose(k[m], ref_k[m], rtol=1e-5)
    grid.close()
