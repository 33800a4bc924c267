"""Batched traces: many grids in one persistent launch (rt_batch_*).

Each grid's result in the mix must equal the same grid traced alone: counts
per level and the created-set checksum bit-exact, photon budget and k_ph /
Gamma equal up to the order of the floating-point sums; graph-replayed
coupled steps equal the same steps taken one grid at a time.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

SUM_ORDER_TOL = {"fp64": 1e-12, "fp32_mixed": 2e-5}


def _grids(seed=7, n=6):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.choice([16, 24, 32, 40]))
        box = synth.box_cm(N)
        pos, ndot, e, sg = synth.random_sources((N, N, N), box / N, int(rng.integers(1, 12)), 1e47, 1e50, rng)
        g = synth._grid(N, box, synth.lognormal_density(N, mean=4e-3, seed=seed * 100 + i), 1.0, pos, ndot, e, sg)
        g["x_HI"] = rng.uniform(0.0, 1.0, N ** 3)
        g["x_HII"] = 1.0 - g["x_HI"]
        out.append(g)
    out.append(synth.stromgren(32))
    return out


def _compare(b, r, b_ref, r_ref, tol):
    np.testing.assert_array_equal(b["counts"], b_ref["counts"])
    np.testing.assert_array_equal(b["hashes"], b_ref["hashes"])
    for key in ("emitted", "absorbed", "escaped"):
        assert abs(b[key] - b_ref[key]) <= 1e-12 * b_ref["emitted"], key
    for key in ("kph", "gamma"):
        ref = r_ref[key]
        m = np.abs(ref) > 1e-8 * np.abs(ref).max() if np.abs(ref).max() > 0 else ref != 0
        np.testing.assert_allclose(r[key][m], ref[m], rtol=tol)


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_batch_equals_each_grid_alone(precision):
    ctx = parity.ctx()
    gs = _grids()
    alone = []
    for g in gs:
        grid = native.Grid(ctx, g, precision)
        alone.append((grid.trace(checksums=True, **synth.DEFAULT_PARAMS), grid.rates()))
        grid.close()
    batch = native.Batch(ctx)
    grids = [native.Grid(ctx, g, precision) for g in gs]
    slots = [batch.add(gr) for gr in grids]
    batch.trace(checksums=True, **synth.DEFAULT_PARAMS)
    for s, gr, (b_ref, r_ref) in zip(slots, grids, alone):
        _compare(batch.budget(s), gr.rates(), b_ref, r_ref, SUM_ORDER_TOL[precision])
    # one grid of the mix against the oracle
    o = parity.run_oracle(gs[0])
    parity.assert_trace_parity(gs[0], batch.budget(slots[0]), grids[0].rates(), o, precision)
    batch.close()


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_batch_graph_steps_equal_single_steps(precision):
    ctx = parity.ctx()
    gs = _grids(seed=11, n=4)
    dt = 0.5 * synth.MYR_S
    ref = []
    for g in gs:
        grid = native.Grid(ctx, g, precision)
        for _ in range(5):
            grid.trace(**synth.DEFAULT_PARAMS)
            grid.chem(dt, 10, synth.ALPHA_B)
        ref.append(grid.rates()["x_HI"])
        grid.close()
    batch = native.Batch(ctx)
    grids = [native.Grid(ctx, g, precision) for g in gs]
    for gr in grids:
        batch.add(gr)
    batch.step(5, dt, 10, synth.ALPHA_B, **synth.DEFAULT_PARAMS)
    tol = 1e-9 if precision == "fp64" else 1e-4
    for gr, x_ref in zip(grids, ref):
        np.testing.assert_allclose(gr.rates()["x_HI"], x_ref, rtol=tol, atol=1e-12)
    batch.close()


def test_batch_remove_add_and_autotune():
    ctx = parity.ctx()
    gs = _grids(seed=5, n=5)
    batch = native.Batch(ctx)
    grids = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    slots = [batch.add(gr) for gr in grids]
    batch.remove(slots[1])
    extra = synth.clumpy(N=24, nsrc=7, seed=77)
    ge = native.Grid(ctx, extra, "fp32_mixed")
    s_new = batch.add(ge)
    assert s_new == slots[1]  # the freed slot is reused
    assert native.rt_batch_size(batch.h) == len(gs)
    params = native.trace_params(checksums=True, **synth.DEFAULT_PARAMS)
    params = native.rt_batch_autotune(batch.h, params)
    assert params.segs_per_iter in (4, 8, 16, 32, 64) and params.blocks_per_sm >= 1
    native.rt_batch_trace(batch.h, params)
    members = [(slots[0], gs[0], grids[0]), (s_new, extra, ge), (slots[3], gs[3], grids[3])]
    for slot, g, gr in members:
        alone = native.Grid(ctx, g, "fp32_mixed")
        b_ref = alone.trace(checksums=True, **synth.DEFAULT_PARAMS)
        _compare(batch.budget(slot), gr.rates(), b_ref, alone.rates(), SUM_ORDER_TOL["fp32_mixed"])
        alone.close()
    batch.close()


def test_a_grid_is_in_one_batch_and_leaves_it_when_destroyed():
    ctx = parity.ctx()
    gs = _grids(seed=9, n=3)
    b1, b2 = native.Batch(ctx), native.Batch(ctx)
    grids = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    slots = [b1.add(gr) for gr in grids]
    for b in (b1, b2):
        with pytest.raises(native.RtError):
            b.add(grids[0])  # already a member of b1
    b1.trace(checksums=True, **synth.DEFAULT_PARAMS)
    grids[1].close()  # destroying a member takes it out of its batch
    b1.grids.pop(slots[1])
    assert native.rt_batch_size(b1.h) == len(gs) - 1
    b1.trace(checksums=True, **synth.DEFAULT_PARAMS)
    for i in (0, 2, 3):
        alone = native.Grid(ctx, gs[i], "fp32_mixed")
        b_ref = alone.trace(checksums=True, **synth.DEFAULT_PARAMS)
        _compare(b1.budget(slots[i]), grids[i].rates(), b_ref, alone.rates(), SUM_ORDER_TOL["fp32_mixed"])
        alone.close()
    b1.remove(slots[0])
    s0 = b2.add(grids[0])  # free to join another batch once removed
    b2.trace(checksums=True, **synth.DEFAULT_PARAMS)
    alone = native.Grid(ctx, gs[0], "fp32_mixed")
    b_ref = alone.trace(checksums=True, **synth.DEFAULT_PARAMS)
    _compare(b2.budget(s0), grids[0].rates(), b_ref, alone.rates(), SUM_ORDER_TOL["fp32_mixed"])
    alone.close()
    b1.close()  # members outlive their batch
    grids[2].trace(**synth.DEFAULT_PARAMS)
    for gr in grids:
        gr.close()
    b2.close()


def test_batch_on_a_non_blocking_stream_orders_member_work():
    """A batch on a caller's non-blocking stream sees state set on its grids' streams."""
    import torch
    ctx = parity.ctx()
    gs = _grids(seed=13, n=3)
    dt = 0.5 * synth.MYR_S
    x_new = [np.random.default_rng(i).uniform(0.0, 1.0, len(g["x_HI"])) for i, g in enumerate(gs)]
    ref = []
    for g, x in zip(gs, x_new):
        grid = native.Grid(ctx, g, "fp32_mixed")
        native.rt_set_state(grid.h, x)
        for _ in range(2):
            grid.trace(**synth.DEFAULT_PARAMS)
            grid.chem(dt, 10, synth.ALPHA_B)
        ref.append(grid.rates()["x_HI"])
        grid.close()
    stream = torch.cuda.Stream()  # non-blocking: not ordered with the legacy stream
    batch = native.Batch(ctx, stream.cuda_stream)
    grids = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    for gr in grids:
        batch.add(gr)
    batch.step(1, dt, 10, synth.ALPHA_B, **synth.DEFAULT_PARAMS)  # captures the graph
    for gr, x in zip(grids, x_new):
        native.rt_set_state(gr.h, torch.tensor(x, dtype=torch.float64, device="cuda"))
    batch.step(2, dt, 10, synth.ALPHA_B, **synth.DEFAULT_PARAMS)
    for gr, x_ref in zip(grids, ref):
        np.testing.assert_allclose(gr.rates()["x_HI"], x_ref, rtol=1e-4, atol=1e-12)
    batch.close()
