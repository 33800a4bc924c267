"""The trace kernel's waits are bounded (failure detection without a fault).

A self-test flag makes the trace wait for one package that never exists, so
nothing ends it; its idle warps must give up after the no-progress limit and
the trace return RT_ERR_TIMEOUT, within a bounded time, leaving the grid and
the context usable: the next trace on the same grid equals the oracle's.
"""
import time

import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_a_stalled_trace_times_out_and_the_grid_stays_usable(precision):
    g = synth.stromgren(32)
    grid = native.Grid(parity.ctx(), g, precision)
    t0 = time.perf_counter()
    with pytest.raises(native.RtError) as err:
        grid.trace(timeout_s=0.05, selftest_stall=True, **synth.DEFAULT_PARAMS)
    assert err.value.code == native.RT_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    b = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, grid.rates(), o, precision)
    grid.close()
