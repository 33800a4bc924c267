"""A trace partitioned by sources over several grids equals the whole trace.

Two ranks are emulated on one GPU: each traces its share of the sources on a
grid holding the whole medium; the partial rates and budgets are summed (the
all-reduce) and installed with rt_set_rates; counts and checksums are
bit-exact with the single-grid trace, the budget and rates equal up to the
order of the sums, and the ionisation update that follows gives the same
state on every rank as on the single grid.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import shard, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_mixed": 2e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_two_shards_equal_the_whole(precision):
    ctx = parity.ctx()
    g = synth.clumpy(N=24, nsrc=9, seed=31)
    full, b_full, r_full = parity.run_gpu(g, precision)
    parts = [shard.shard_trace(ctx, g, precision, rank, 2, checksums=True, **synth.DEFAULT_PARAMS)
             for rank in range(2)]
    k = parts[0][2] + parts[1][2]  # the all-reduce
    gm = parts[0][3] + parts[1][3]
    f = sum(shard.budget_vector(p[1])[0] for p in parts)
    i = sum(shard.budget_vector(p[1])[1] for p in parts)
    b = shard.budget_from_vector(f, i)
    np.testing.assert_array_equal(b["counts"], b_full["counts"])
    np.testing.assert_array_equal(b["hashes"], b_full["hashes"])
    assert b["segments"] == b_full["segments"]
    for key in ("emitted", "absorbed", "escaped"):
        assert abs(b[key] - b_full[key]) <= 1e-9 * b_full["emitted"]
    ref = np.asarray(r_full["kph"])
    m = ref > 1e-8 * ref.max()
    np.testing.assert_allclose(k.cpu().numpy()[m], ref[m], rtol=TOL[precision])
    dt = 0.5 * synth.MYR_S
    full.chem(dt, 10, synth.ALPHA_B)
    x_full = full.rates()["x_HI"]
    for grid, _, _, _ in parts:
        shard.install(grid, k, gm)
        np.testing.assert_allclose(grid.rates()["kph"], k.double().cpu().numpy(), rtol=1e-7 if precision != "fp64" else 0)
        grid.chem(dt, 10, synth.ALPHA_B)
        np.testing.assert_allclose(grid.rates()["x_HI"], x_full, rtol=1e-9 if precision == "fp64" else 1e-4,
                                   atol=1e-12)
        grid.close()
    full.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_shards_with_packages_in_flight(precision):
    """With a finite speed of light each rank keeps its own sources' packages
    in flight; the summed steps equal the single grid's coupled steps."""
    ctx = parity.ctx()
    g = synth.clumpy(N=20, nsrc=6, seed=37)
    g["x_HI"] = np.full(20 ** 3, 0.02)
    g["x_HII"] = 1.0 - g["x_HI"]
    light = 3.3 * g["box_len_cm"] / 20
    dt = 0.05 * synth.MYR_S
    p = dict(synth.DEFAULT_PARAMS, checksums=True, light_cm=light)
    from paper_1012_2865_gb300 import native
    full = native.Grid(ctx, g, precision)
    ranks = [shard.ShardGrid(ctx, g, precision, r, 2) for r in range(2)]
    for step in range(5):
        b_full = full.trace(**p)
        parts = [rk.trace(**p) for rk in ranks]
        k = parts[0][1] + parts[1][1]
        gm = parts[0][2] + parts[1][2]
        f = sum(shard.budget_vector(q[0])[0] for q in parts)
        i = sum(shard.budget_vector(q[0])[1] for q in parts)
        b = shard.budget_from_vector(f, i)
        np.testing.assert_array_equal(b["counts"], b_full["counts"])
        np.testing.assert_array_equal(b["hashes"], b_full["hashes"])
        for key in ("emitted", "absorbed", "escaped", "resumed", "halted"):
            # the media differ by the update's response to the rates' summation order
            assert abs(b[key] - b_full[key]) <= parity.BUDGET_TOL[precision] * (b_full["emitted"] + b_full["resumed"]), key
        ref = full.rates()["kph"]
        m = ref > 1e-8 * ref.max()
        np.testing.assert_allclose(k.double().cpu().numpy()[m], ref[m], rtol=TOL[precision])
        full.chem(dt, 10, synth.ALPHA_B)
        for rk in ranks:
            rk.install(k, gm)
            rk.chem(dt, 10, synth.ALPHA_B)
    x_full = full.rates()["x_HI"]
    for rk in ranks:
        np.testing.assert_allclose(rk.grid.rates()["x_HI"], x_full, rtol=1e-9 if precision == "fp64" else 1e-4,
                                   atol=1e-12)
        rk.close()
    full.close()
