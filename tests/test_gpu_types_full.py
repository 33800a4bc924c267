"""Photon types at full size: the typed clumpy configuration (128^3, 30
sources cycling through H I, He I and He II ionising, helium absorbers) in
the launch configuration the benchmark's photon_types leg times, against the
oracle element by element (about 3.8e8 segments, 15 s of one CPU core)."""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def typed_and_oracle():
    g = synth.typed_clumpy()
    o = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                     g["sigma_cm2"], src_type=g["types"], n_he=g["n_he"], **synth.DEFAULT_PARAMS)
    return g, o


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_typed_clumpy_128_full(typed_and_oracle, precision):
    g, o = typed_and_oracle
    grid = native.Grid(parity.ctx(), g, precision)
    grid.set_absorbers(g["n_he"][0], g["n_he"][1])
    grid.set_source_types(g["types"])
    b = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    assert b["status"] == 0
    np.testing.assert_array_equal(b["counts"], o["counts"])
    np.testing.assert_array_equal(b["hashes"], o["hashes"])
    if precision == "fp64":
        assert b["segments"] == o["segments"]
    em = o["budget"][0]
    bt = parity.BUDGET_TOL[precision]
    assert abs(b["absorbed"] - o["budget"][1]) <= bt * em and abs(b["escaped"] - o["budget"][2]) <= bt * em
    for t in range(3):
        r = grid.rates_typed(t)
        for key, ref in (("kph", o["kph_types"][t]), ("gamma", o["gamma_types"][t])):
            m = parity.receiving_mask(g, o["kph_types"][t], em) & (ref != 0)
            assert m.sum() > 1000, (t, key)
            rel = np.abs(np.asarray(r[key])[m] - ref[m]) / ref[m]
            assert rel.max() <= parity.TOL[precision], (t, key, float(rel.max()))
    grid.close()
