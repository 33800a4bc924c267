"""FP64 CUDA path vs the FP64 oracle (element by element, through the C ABI)."""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


def test_config0_trace_and_chemistry():
    """32^3 Test-1 medium, corner source, one trace + 10 implicit substeps over 1 Myr."""
    g = synth.stromgren(32)
    grid, b, r = parity.run_gpu(g)
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o)
    grid.chem(1.0 * synth.MYR_S, 10, synth.ALPHA_B)
    x_gpu = grid.rates()["x_HI"]
    z_gpu = grid.x_HII()
    x_o, z_o = oracle.chem(g["n_H"], g["x_HI"], g["x_HII"], o["kph"], synth.MYR_S, 10, synth.ALPHA_B)
    np.testing.assert_allclose(x_gpu, x_o, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(z_gpu, z_o, rtol=1e-6, atol=1e-12)
    grid.close()


@pytest.mark.parametrize("seed,dims,nsrc,level0,phi_c", [
    (0, (24, 24, 24), 6, 1, 5.1),
    (1, (37, 23, 29), 9, 0, 3.1),
    (2, (16, 40, 8), 4, 2, 10.1),
])
def test_clumpy_ragged_grids(seed, dims, nsrc, level0, phi_c):
    rng = np.random.default_rng(seed)
    box = 6.6 * synth.KPC_CM * dims[0] / 32
    dx = box / dims[0]
    n = synth.lognormal_density(None, mean=2e-3, seed=seed, dims=dims)
    pos, ndot, e, sg = synth.random_sources(dims, dx, nsrc, 1e48, 1e50, rng)
    g = synth._grid(dims, box, n, rng.uniform(0.0, 1.0, int(np.prod(dims))), pos, ndot, e, sg)
    _, b, r = parity.run_gpu(g, level0=level0, phi_c=phi_c)
    o = parity.run_oracle(g, level0=level0, phi_c=phi_c)
    parity.assert_trace_parity(g, b, r, o)


def test_partially_ionised_128():
    """128^3 with an ionised octant sphere of 90 cells (state near t = 500 Myr)."""
    N = 128
    g = synth.stromgren(N)
    i = np.arange(N) + 0.5
    rad = np.sqrt(i[None, None, :] ** 2 + i[None, :, None] ** 2 + i[:, None, None] ** 2).reshape(-1)
    x = 1.0 / (1.0 + np.exp(-(rad - 90.0) / 2.0))
    g["x_HI"] = np.clip(x, 1e-6, 1.0)
    g["x_HII"] = 1.0 - g["x_HI"]
    _, b, r = parity.run_gpu(g)
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o)


def test_edge_cases():
    ctx = parity.ctx()
    # no sources: all zero
    g = synth.stromgren(8)
    grid = native.Grid(ctx, dict(g, ndot=np.zeros(0), pos_cm=np.zeros((0, 3)), e_ph_eV=np.zeros(0),
                                 sigma_cm2=np.zeros(0)))
    b = grid.trace()
    assert b["emitted"] == 0 and b["counts"].sum() == 0
    assert np.all(grid.rates()["kph"] == 0)
    grid.close()
    # one-cell grid, source on the far corner, transparent medium
    g = synth.stromgren(1)
    g["n_H"] = np.zeros(1)
    g["pos_cm"] = np.array([[g["box_len_cm"]] * 3])
    _, b, r = parity.run_gpu(g)
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o)
    # no splitting at all (max_level = level0), and level0 = 0
    g = synth.clumpy(N=16, nsrc=3, seed=5)
    for kw in (dict(max_level=1), dict(level0=0, max_level=0), dict(level0=0, phi_c=25.1)):
        _, b, r = parity.run_gpu(g, **kw)
        o = parity.run_oracle(g, **kw)
        parity.assert_trace_parity(g, b, r, o)


def test_queue_overflow_retry_and_async_error():
    g = synth.stromgren(32)
    o = parity.run_oracle(g)
    grid = native.Grid(parity.ctx(), g)
    # explicit tiny capacity, asynchronous: the overflow is reported, not hidden
    grid.trace(sync=False, queue_capacity=64)
    with pytest.raises(native.RtError) as e:
        native.rt_get_budget(grid.h)
    assert e.value.code == native.RT_ERR_QUEUE_OVERFLOW
    # the grid stays usable; an automatic capacity grows and the result is exact
    b = grid.trace()
    assert b["status"] == 0
    np.testing.assert_array_equal(b["counts"], o["counts"])
    grid.close()


def test_invalid_arguments_are_rejected():
    ctx = parity.ctx()
    g = synth.stromgren(4)
    with pytest.raises(native.RtError) as e:
        native.rt_create_grid(ctx, (4, 4, 0), g["box_len_cm"], g["n_H"], g["x_HI"])
    assert e.value.code == native.RT_ERR_INVALID_ARG
    bad = g["x_HI"].copy()
    bad[3] = 1.5
    with pytest.raises(native.RtError):
        native.rt_create_grid(ctx, (4, 4, 4), g["box_len_cm"], g["n_H"], bad)
    grid = native.Grid(ctx, g)
    before = grid.rates()["x_HI"]
    for arr, name in ((np.where(np.arange(64) == 17, -0.25, g["x_HI"]), "x_HI[17]"),
                      (np.where(np.arange(64) == 5, np.nan, g["x_HI"]), "x_HI[5]")):
        with pytest.raises(native.RtError) as e:
            native.rt_set_state(grid.h, arr)
        assert e.value.code == native.RT_ERR_INVALID_ARG and name in str(e.value)
    n_bad = g["n_H"].copy()
    n_bad[40] = np.inf
    with pytest.raises(native.RtError) as e:
        native.rt_set_state(grid.h, g["x_HI"], n_H=n_bad)
    assert "n_H[40]" in str(e.value)
    np.testing.assert_array_equal(grid.rates()["x_HI"], before)  # a rejected state changes nothing
    with pytest.raises(native.RtError):
        native.rt_add_sources(grid.h, [[-1.0, 0, 0]], [1e48], [13.6], [6.3e-18])
    with pytest.raises(native.RtError):
        grid.trace(phi_c=-1.0)
    with pytest.raises(native.RtError):
        grid.trace(level0=3, max_level=2)
    grid.close()


def test_stromgren_500myr_fp64():
    """Coupled 128^3 evolution, 1000 steps of 0.5 Myr: R_IF reaches R_s within 2 %."""
    N = 128
    g = synth.stromgren(N)
    grid = native.Grid(parity.ctx(), g)
    V = (g["box_len_cm"] / N) ** 3
    rs = (3 * 5e48 / (4 * np.pi * synth.ALPHA_B * 1e-3 ** 2)) ** (1 / 3)
    trec = 1 / (synth.ALPHA_B * 1e-3)
    dt = 0.5 * synth.MYR_S
    for s in range(1000):
        grid.trace(sync=False, queue_capacity=1 << 22)
        grid.chem(dt, 10, synth.ALPHA_B)
        if (s + 1) % 200 == 0:
            b = native.rt_get_budget(grid.h)
            assert abs(b["emitted"] - b["absorbed"] - b["escaped"]) <= 1e-12 * b["emitted"]
            t = (s + 1) * dt
            R = (6 * np.sum(grid.x_HII()) * V / np.pi) ** (1 / 3)
            ana = rs * (1 - np.exp(-t / trec)) ** (1 / 3)
            assert 0.97 < R / ana < 1.035, (t, R / ana)
    assert abs(R / rs - 1) < 0.02, R / rs
    grid.close()


def test_long_trace_with_a_short_no_progress_limit():
    """A trace several times longer than the no-progress limit completes: the
    limit applies to a warp's idle stretch without any change of the
    outstanding count, not to the trace (a warp that has been busy starts a
    new stretch)."""
    g = synth.stromgren_snapshot(256)
    grid = native.Grid(parity.ctx(), g, "fp64")
    b = grid.trace(timeout_s=0.01, **synth.DEFAULT_PARAMS)
    assert b["status"] == 0
    assert b["kernel_ms"] > 20.0  # the trace outlasts the 10 ms limit (about 30 ms on a GB300)
    assert abs(b["emitted"] - b["absorbed"] - b["escaped"]) <= 1e-12 * b["emitted"]
    grid.close()
