"""The largest package tree a serving request can make, in one launch.

A fully ionised 256^3 box (x_HI = 1e-4: about 0.1 optical depths across
it) with 500 sources: no package terminates, every ray walks to the box
boundary and splits at each R_split(l) on the way (Eq. split), so each
source's tree reaches level 9-10.  The automatically sized queue holds every
record of that tree (32 bytes each on the mixed path), so the trace runs as
one launch.  Checked at this size by properties that hold at any size:

* one launch (passes == 1, status 0);
* the same trace in four passes over ranges of the sources creates the same
  packages (per-level counts, checksums) and segments, with budgets equal up
  to the order of the sums;
* photon conservation: emitted = absorbed + escaped (Sec. 2.2), and the
  deposits add up to the photons absorbed.

With -s it prints the per-level counts and the share of the largest level,
which is the least a queue of recycled slots would have to hold at once:
packages are taken up in ticket (breadth-first) order, so when the first
package of level l + 1 is taken up the children of every package of level l
that has finished are waiting in the queue.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, NSRC, X_HI = 256, 500, 1e-4


def test_fully_ionised_256_with_500_sources_in_one_launch():
    free, _ = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip(f"needs ~70 GB of device memory for the queue ({free / 1e9:.0f} GB free)")
    g = synth.clumpy(N, NSRC)
    g["x_HI"] = np.full(N ** 3, X_HI)
    g["x_HII"] = 1.0 - g["x_HI"]
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    one = grid.trace(**p)
    assert one["status"] == 0 and one["passes"] == 1
    assert one["queue_peak"] <= 1 << 31
    assert one["absorbed"] + one["escaped"] == pytest.approx(one["emitted"], rel=1e-9)
    k1 = grid.rates()["kph"]
    # what the deposits add up to is what the packages lost (Eqs. flux, kph):
    # sum_c k_c n_HI,c V = absorbed, to the FP32 rounding of the deposits
    dx = g["box_len_cm"] / N
    dep = float(np.sum(k1 * (g["n_H"] * g["x_HI"]))) * dx ** 3
    assert abs(dep - one["absorbed"]) <= 1e-5 * one["emitted"], (dep, one["absorbed"], one["emitted"])
    counts = np.asarray(one["counts"], dtype=np.int64)
    kids = int(counts[p["level0"] + 1:].sum())
    assert one["queue_peak"] <= kids // 4 * 3  # at most children 1-3 of every split
    four = grid.trace(passes=4, **p)
    assert four["status"] == 0 and four["passes"] == 4
    np.testing.assert_array_equal(four["counts"], one["counts"])
    np.testing.assert_array_equal(four["hashes"], one["hashes"])
    assert four["segments"] == one["segments"]
    for key in ("absorbed", "escaped"):
        assert four[key] == pytest.approx(one[key], rel=1e-9)
    k4 = grid.rates()["kph"]
    # the same trace again in one launch, with the queue it now holds and the
    # segments per queue visit chosen from the first trace's package length
    again = grid.trace(**p)
    assert again["status"] == 0 and again["passes"] == 1
    np.testing.assert_array_equal(again["counts"], one["counts"])
    np.testing.assert_array_equal(again["hashes"], one["hashes"])
    assert again["segments"] == one["segments"]
    grid.close()
    levels = {l: int(c) for l, c in enumerate(counts) if c}
    per_cell = one["segments"] / N ** 3
    print(f"\nfully ionised {N}^3, {NSRC} sources: {one['segments']:.4g} segments "
          f"({per_cell:.0f} per cell), {int(counts.sum()):.4g} packages, {one['queue_peak']:.4g} queue "
          f"records ({one['queue_peak'] * 32 / 1e9:.1f} GB), one launch {one['kernel_ms']:.1f} ms "
          f"(again: {again['kernel_ms']:.1f} ms), "
          f"four passes {four['kernel_ms']:.1f} ms (largest pass {four['queue_peak']:.4g} records)")
    print("packages per level:", levels)
    print(f"largest level: {max(levels.values()) / kids:.3f} of all children")
    # k_ph: the same deposits added in another order.  n positive FP32 terms
    # summed in two orders differ by at most (n - 1) 2^-24 of their sum; a
    # cell here takes about as many deposits as there are segments per cell
    # (~8,500: every source's rays cross it): rtol = 5e-4.
    m = k1 > 1e-8 * k1.max()
    np.testing.assert_allclose(k4[m], k1[m], rtol=5e-4)
    assert abs(k4.sum() - k1.sum()) <= 1e-6 * k1.sum()
