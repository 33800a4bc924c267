"""State upload and rate read-back without waiting (rt_set_state_async,
rt_get_rates_async, rt_wait_rates), through the C ABI on the GPU.

The asynchronous calls must leave the grid exactly as the synchronous ones do
(the same state, the same trace), reject a bad state on the device without
changing anything, and report the rejection once; read-backs must equal
rt_get_rates."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1012_2865_gb300 import build, native
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = native.rt_ctx_create(0)
    yield c
    native.rt_ctx_destroy(c)


def _pinned(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype).pin_memory()


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_async_state_equals_sync_state(ctx, precision):
    from paper_1012_2865_gb300 import native, synth
    g = synth.stromgren_snapshot(64)
    snap_x, snap_z = g["x_HI"], g["x_HII"]
    neutral = dict(g, x_HI=np.ones_like(snap_x), x_HII=np.zeros_like(snap_z))
    a = native.Grid(ctx, neutral, precision)
    b = native.Grid(ctx, neutral, precision)
    native.rt_set_state(a.h, snap_x, snap_z)
    hx, hz = _pinned(snap_x), _pinned(snap_z)
    native.rt_set_state_async(b.h, hx, hz)
    native.rt_synchronize(b.h)
    ra, rb = a.rates(), b.rates()
    assert np.array_equal(ra["x_HI"], rb["x_HI"])
    assert np.array_equal(a.x_HII(), b.x_HII())
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    ba, bb = a.trace(**p), b.trace(**p)
    assert np.array_equal(ba["counts"], bb["counts"]) and np.array_equal(ba["hashes"], bb["hashes"])
    assert ba["segments"] == bb["segments"]
    # device arrays, and x_HII left to the complement
    c = native.Grid(ctx, neutral, precision)
    native.rt_set_state_async(c.h, torch.tensor(snap_x, dtype=torch.float64, device="cuda"))
    native.rt_synchronize(c.h)
    assert np.array_equal(c.rates()["x_HI"], snap_x)
    assert np.array_equal(c.x_HII(), 1.0 - snap_x)
    for gr in (a, b, c):
        gr.close()


def test_rejected_async_state_changes_nothing_and_is_reported_once(ctx):
    from paper_1012_2865_gb300 import native, synth
    g = synth.stromgren(32)
    grid = native.Grid(ctx, g, "fp32_mixed")
    good = np.full(grid.ncell, 0.25)
    native.rt_set_state_async(grid.h, _pinned(good))
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    before = grid.trace(**p)
    z_before = grid.x_HII()
    bad = good.copy()
    bad[1234] = 1.5
    native.rt_set_state_async(grid.h, _pinned(bad))
    with pytest.raises(native.RtError) as ei:
        native.rt_synchronize(grid.h)
    assert ei.value.code == native.RT_ERR_INVALID_ARG and "x_HI[1234]" in str(ei.value)
    assert np.array_equal(grid.rates()["x_HI"], good)
    assert np.array_equal(grid.x_HII(), z_before)
    native.rt_synchronize(grid.h)  # reported once
    # the absorber density was restored too: the same trace as before the rejected upload
    after = grid.trace(**p)
    assert after["segments"] == before["segments"]
    assert np.array_equal(after["counts"], before["counts"]) and np.array_equal(after["hashes"], before["hashes"])
    # a rejection is also the status of the next trace, which still runs on the kept state
    bad_n = np.full(grid.ncell, 1e-3)
    bad_n[7] = -1.0
    native.rt_set_state_async(grid.h, _pinned(good), n_H=_pinned(bad_n))
    with pytest.raises(native.RtError) as ei:
        grid.trace(**synth.DEFAULT_PARAMS)
    assert ei.value.code == native.RT_ERR_INVALID_ARG and "n_H[7]" in str(ei.value)
    b = grid.trace(**synth.DEFAULT_PARAMS)
    assert b["status"] == 0
    native.rt_synchronize(grid.h)
    grid.close()


def test_async_read_back_equals_sync_read_back(ctx):
    from paper_1012_2865_gb300 import native, synth
    g = synth.stromgren_snapshot(64)
    grid = native.Grid(ctx, g, "fp32_mixed")
    grid.trace(**synth.DEFAULT_PARAMS)
    grid.chem(synth.MYR_S, 10, synth.ALPHA_B)
    ref = grid.rates()
    n = grid.ncell
    hk = torch.empty(n, dtype=torch.float64).pin_memory()
    hg = torch.empty(n, dtype=torch.float64).pin_memory()
    hx = torch.empty(n, dtype=torch.float64).pin_memory()
    native.rt_get_rates_async(grid.h, hk, hg, hx, native.RT_DTYPE_F64)
    native.rt_wait_rates(grid.h)
    assert np.array_equal(hk.numpy(), ref["kph"]) and np.array_equal(hg.numpy(), ref["gamma"])
    assert np.array_equal(hx.numpy(), ref["x_HI"])
    k32 = torch.empty(n, dtype=torch.float32).pin_memory()
    native.rt_get_rates_async(grid.h, kph=k32, dtype=native.RT_DTYPE_F32)
    dk = torch.empty(n, dtype=torch.float32, device="cuda")
    native.rt_get_rates_async(grid.h, kph=dk, dtype=native.RT_DTYPE_F32)
    native.rt_synchronize(grid.h)
    assert np.array_equal(k32.numpy(), ref["kph"].astype(np.float32))
    assert np.array_equal(dk.cpu().numpy(), ref["kph"].astype(np.float32))
    with pytest.raises(ValueError):
        native.rt_get_rates_async(grid.h, kph=np.empty(n, dtype=np.float32), dtype=native.RT_DTYPE_F64)
    grid.close()


def test_pipelined_steps_equal_sequential_steps(ctx):
    """Three coupled steps with uploads and read-backs overlapping the next
    step's kernels give the same per-step results as synchronous calls."""
    from paper_1012_2865_gb300 import native, synth
    g = synth.stromgren_snapshot(64)
    dt = 0.5 * synth.MYR_S
    states = [g["x_HI"], np.clip(g["x_HI"] * 0.9, 0, 1), np.clip(g["x_HI"] * 1.1, 0, 1)]
    seq = native.Grid(ctx, g, "fp32_mixed")
    want = []
    for x in states:
        native.rt_set_state(seq.h, x)
        seq.trace(**synth.DEFAULT_PARAMS)
        seq.chem(dt, 10, synth.ALPHA_B)
        r = seq.rates()
        want.append((r["kph"], r["x_HI"]))
    seq.close()
    pipe = native.Grid(ctx, g, "fp32_mixed")
    pipe.trace(**synth.DEFAULT_PARAMS)  # sizes the queue
    n = pipe.ncell
    ins = [_pinned(x) for x in states]
    outs = [(torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory())
            for _ in states]
    for i, x in enumerate(ins):
        native.rt_set_state_async(pipe.h, x)
        pipe.trace(sync=False, **synth.DEFAULT_PARAMS)
        pipe.chem(dt, 10, synth.ALPHA_B)
        native.rt_wait_rates(pipe.h)
        native.rt_get_rates_async(pipe.h, kph=outs[i][0], x_HI=outs[i][1])
    native.rt_synchronize(pipe.h)
    for (k, x), (hk, hx) in zip(want, outs):
        m = k > 1e-8 * k.max()
        assert np.max(np.abs(hk.numpy()[m] - k[m]) / k[m]) < 1e-5
        assert np.allclose(hx.numpy(), x, rtol=1e-5, atol=1e-12)
    pipe.close()
