"""Covering-factor correction (Sec. 2.3) on the GPU vs the oracle.

With RT_TRACE_FC both CUDA paths scale each segment's k_ph and Gamma
contribution by f_c; counts, checksums and the photon budget stay those of
the uncorrected trace, and k_ph / Gamma match the oracle run with the same
correction within the paths' tolerances.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import synth

pytestmark = pytest.mark.gpu


def _cases():
    g1 = synth.stromgren(32)
    g2 = synth.clumpy(N=24, nsrc=6, seed=9)
    g3 = synth.clumpy(N=20, nsrc=4, seed=12)
    g3["x_HI"] = np.random.default_rng(4).uniform(0.0, 0.2, 20 ** 3)  # mostly ionised: long rays
    g3["x_HII"] = 1.0 - g3["x_HI"]
    return [("stromgren32", g1), ("clumpy24", g2), ("ionised20", g3)]


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("name,g", _cases())
def test_fc_matches_oracle(precision, name, g):
    o = parity.run_oracle(g, fc=True)
    grid, b, r = parity.run_gpu(g, precision, fc=True)
    parity.assert_trace_parity(g, b, r, o, precision)
    b0 = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)  # the same grid without the correction
    for key in ("emitted", "absorbed", "escaped"):
        assert abs(b[key] - b0[key]) <= 1e-9 * b0["emitted"]
    np.testing.assert_array_equal(b["counts"], b0["counts"])
    grid.close()
