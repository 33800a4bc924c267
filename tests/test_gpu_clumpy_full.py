"""Full-size clumpy multi-source trace (256^3, 1000 sources) vs the oracle.

The oracle traces the whole configuration (about 1.5e8 segments, ~10 s of
one CPU core), so the comparison is element by element at full size.
"""
import pytest

import parity
from paper_1012_2865_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clumpy_and_oracle():
    g = synth.clumpy()
    return g, parity.run_oracle(g)


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_clumpy_256_full(clumpy_and_oracle, precision):
    g, o = clumpy_and_oracle
    grid, b, r = parity.run_gpu(g, precision)
    worst = parity.assert_trace_parity(g, b, r, o, precision)
    print(f"clumpy 256^3 {precision}: largest relative error against the oracle", worst)
    assert b["fallbacks"] < 1e-3 * b["segments"]
    grid.close()
