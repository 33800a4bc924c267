"""Adaptive RT timestep (Sec. 3.4) on the GPU vs the oracle.

The GPU evaluates the per-cell timestep and the smoothing in FP32 (the
front test in FP64); the result matches the oracle's FP64 value to 1e-5 on
states with a real ionisation front, given the rates this grid's own trace
deposited.
"""
import numpy as np
import pytest

import parity
from oracle import timestep
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


def _oracle(grid, g, r, **kw):
    return timestep.rt_timestep(tuple(g["dims"]), g["box_len_cm"] / g["dims"][0], g["n_H"], r["x_HI"],
                                np.asarray(r["kph"], dtype=np.float64), **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("case", ["snapshot64", "clumpy24"])
def test_timestep_matches_oracle(precision, case):
    g = synth.stromgren_snapshot(64) if case == "snapshot64" else synth.clumpy(N=24, nsrc=6, seed=9)
    grid, b, r = parity.run_gpu(g, precision)
    for kw in (dict(eps_ion=0.05, dt_max=1e16), dict(eps_ion=0.1, dt_max=float("inf"), tau_front=2.0),
               dict(eps_ion=0.05, dt_max=1e16, dt_prev=1e9)):
        dt_gpu = native.rt_timestep(grid.h, **kw)
        dt_o = _oracle(grid, g, r, **kw)
        assert dt_gpu == pytest.approx(dt_o, rel=1e-5), (kw, dt_gpu, dt_o)
    grid.close()


def test_no_front_gives_dt_max():
    g = synth.stromgren(16)
    g["x_HI"] = np.full(16 ** 3, 1e-9)
    g["x_HII"] = 1.0 - g["x_HI"]
    grid, b, r = parity.run_gpu(g, "fp32_mixed")
    assert native.rt_timestep(grid.h, dt_max=3e15) == 3e15
    assert native.rt_timestep(grid.h) == float("inf")
    grid.close()
