"""Traces split into passes over ranges of the sources.

A trace whose packages do not fit the queue at once runs as several launches
over equal ranges of the sources, adding into the same k_ph, Gamma and photon
budget.  Splitting changes only the order of the floating-point sums: the
created packages (counts per level, checksum) and segments are identical, and
each pass reuses the queue, so a queue that holds one pass's packages but not
the whole trace's suffices.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

SUM_ORDER_TOL = {"fp64": 1e-12, "fp32_mixed": 2e-5}


def _grid(seed=21, N=40, nsrc=12):
    rng = np.random.default_rng(seed)
    box = synth.box_cm(N)
    pos, ndot, e, sg = synth.random_sources((N, N, N), box / N, nsrc, 1e48, 1e50, rng)
    g = synth._grid(N, box, synth.lognormal_density(N, mean=2e-3, seed=seed), 1.0, pos, ndot, e, sg)
    g["x_HI"] = rng.uniform(0.0, 0.3, N ** 3)  # mostly ionised: long rays, deep trees
    g["x_HII"] = 1.0 - g["x_HI"]
    return g


def _same(b, r, b_ref, r_ref, tol):
    np.testing.assert_array_equal(b["counts"], b_ref["counts"])
    np.testing.assert_array_equal(b["hashes"], b_ref["hashes"])
    assert b["segments"] == b_ref["segments"]
    for key in ("emitted", "absorbed", "escaped"):
        assert abs(b[key] - b_ref[key]) <= 1e-12 * b_ref["emitted"], key
    for key in ("kph", "gamma"):
        ref = r_ref[key]
        m = np.abs(ref) > 1e-8 * np.abs(ref).max()
        np.testing.assert_allclose(r[key][m], ref[m], rtol=tol)
        assert np.all(r[key][~m] <= 1e-7 * np.abs(ref).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_passes_equal_one_launch_and_the_oracle(precision):
    g = _grid()
    grid, b1, r1 = parity.run_gpu(g, precision)
    assert b1["passes"] == 1 and b1["queue_peak"] == b1["queue_pushed"]
    for passes in (3, 12, 50):  # 50 > sources: one pass per source
        b = grid.trace(checksums=True, passes=passes, **synth.DEFAULT_PARAMS)
        assert b["passes"] == min(passes, 12)
        # the same packages (how many of them pass through the queue depends
        # on scheduling: children placed in a free lane of the warp do not)
        np.testing.assert_array_equal(b["counts"], b1["counts"])
        assert b["queue_peak"] < b1["queue_peak"]
        _same(b, grid.rates(), b1, r1, SUM_ORDER_TOL[precision])
    b = grid.trace(checksums=True, passes=3, **synth.DEFAULT_PARAMS)
    parity.assert_trace_parity(g, b, grid.rates(), parity.run_oracle(g), precision)
    # a caller's minimum holds for its own call only
    assert grid.trace(**synth.DEFAULT_PARAMS)["passes"] == 1
    grid.close()


def test_a_queue_for_one_pass_suffices():
    g = _grid(seed=22)
    grid, b1, r1 = parity.run_gpu(g, "fp32_mixed")
    b4 = grid.trace(checksums=True, passes=4, **synth.DEFAULT_PARAMS)
    grid.close()
    # queue use varies a little from run to run (children placed in a free
    # lane of the splitting warp skip the queue): keep a margin both ways
    cap = b4["queue_peak"] * 3 // 2 + 64
    assert cap < b1["queue_peak"] * 3 // 4
    fresh = native.Grid(parity.ctx(), g, "fp32_mixed")  # its queue is allocated at `cap`
    with pytest.raises(native.RtError) as e:  # one launch overflows this queue ...
        fresh.trace(checksums=True, queue_capacity=cap, **synth.DEFAULT_PARAMS)
    assert e.value.code == native.RT_ERR_QUEUE_OVERFLOW
    # ... four passes fit, and equal the one-launch trace
    b = fresh.trace(checksums=True, queue_capacity=cap, passes=4, **synth.DEFAULT_PARAMS)
    _same(b, fresh.rates(), b1, r1, SUM_ORDER_TOL["fp32_mixed"])
    fresh.close()


def test_batch_passes_and_graph_steps():
    ctx = parity.ctx()
    gs = [_grid(seed=30 + i, N=24 + 8 * i, nsrc=3 + 2 * i) for i in range(4)]
    dt = 0.5 * synth.MYR_S
    alone = []
    for g in gs:
        grid = native.Grid(ctx, g, "fp32_mixed")
        alone.append((grid.trace(checksums=True, **synth.DEFAULT_PARAMS), grid.rates()))
        grid.close()
    batch = native.Batch(ctx)
    grids = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    slots = [batch.add(gr) for gr in grids]
    batch.trace(checksums=True, passes=5, **synth.DEFAULT_PARAMS)
    for s, gr, (b_ref, r_ref) in zip(slots, grids, alone):
        b = batch.budget(s)
        assert b["passes"] == 5
        _same(b, gr.rates(), b_ref, r_ref, SUM_ORDER_TOL["fp32_mixed"])
    batch.trace(**synth.DEFAULT_PARAMS)
    assert batch.budget(slots[0])["passes"] == 1
    # graph steps with passes equal graph steps without
    ref = []
    for g in gs:
        grid = native.Grid(ctx, g, "fp32_mixed")
        for _ in range(3):
            grid.trace(**synth.DEFAULT_PARAMS)
            grid.chem(dt, 10, synth.ALPHA_B)
        ref.append(grid.rates()["x_HI"])
        grid.close()
    batch2 = native.Batch(ctx)
    grids2 = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    for gr in grids2:
        batch2.add(gr)
    batch2.step(3, dt, 10, synth.ALPHA_B, passes=4, **synth.DEFAULT_PARAMS)
    for gr, x_ref in zip(grids2, ref):
        np.testing.assert_allclose(gr.rates()["x_HI"], x_ref, rtol=1e-4, atol=1e-12)
    batch.close()
    batch2.close()
