"""Photon types on the GPU (Sec. 3.2) against the oracle.

Sources of the three types (H I, He I, He II ionising) share one trace; each
type's packages are absorbed by their own species.  Compared with the
oracle: packages per level and the created-set checksum bit-exact, segments
exact on the FP64 path, the photon budget, and each type's k_ph and Gamma
within the parity tolerances; then the same in a batch and with a finite
speed of light.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

E_ION = (13.6, 24.6, 54.4)


def _typed(N=32, nsrc=12, seed=41):
    g = synth.clumpy(N=N, nsrc=nsrc, seed=seed)
    g["x_HI"] = np.full(N ** 3, 0.05)
    g["x_HII"] = 1.0 - g["x_HI"]
    rng = np.random.default_rng(seed + 1)
    n = N ** 3
    he = np.stack([synth.round_f32(0.08 * g["n_H"] * rng.uniform(0.2, 1.0, n)),
                   synth.round_f32(0.02 * g["n_H"] * rng.uniform(0.0, 1.0, n))])
    types = np.arange(nsrc) % 3
    g["e_ph_eV"] = np.array([E_ION[t] + 2.0 + 1.5 * k for k, t in enumerate(types)])
    return g, he, types


def _grid(g, he, types, precision, stream=None):
    grid = native.Grid(parity.ctx(), g, precision, stream=stream)
    grid.set_absorbers(he[0], he[1])
    grid.set_source_types(types)
    return grid


def _compare(g, b, grid, o, precision, exact_segments=None):
    assert b["status"] == 0
    np.testing.assert_array_equal(b["counts"], o["counts"])
    np.testing.assert_array_equal(b["hashes"], o["hashes"])
    if exact_segments if exact_segments is not None else precision == "fp64":
        assert b["segments"] == o["segments"]
    em = o["budget"][0]
    bt = parity.BUDGET_TOL[precision]
    assert abs(b["emitted"] - em) <= bt * em
    assert abs(b["absorbed"] - o["budget"][1]) <= bt * em
    assert abs(b["escaped"] - o["budget"][2]) <= bt * em
    for t in range(3):
        r = grid.rates_typed(t)
        ref_k, ref_g = o["kph_types"][t], o["gamma_types"][t]
        mask = parity.receiving_mask(g, ref_k, em)
        for got, ref, key in ((r["kph"], ref_k, "kph"), (r["gamma"], ref_g, "gamma")):
            ref, got = ref[mask], np.asarray(got)[mask]
            nz = ref != 0
            assert nz.sum() > 10, (t, key)
            rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
            assert rel.max() <= parity.TOL[precision], (t, key, float(rel.max()))


def _oracle(g, he, types, **kw):
    p = dict(synth.DEFAULT_PARAMS)
    p.update(kw)
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], src_type=types, n_he=he, **p)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_typed_sources_match_the_oracle(precision):
    g, he, types = _typed()
    grid = _grid(g, he, types, precision)
    b = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    o = _oracle(g, he, types)
    _compare(g, b, grid, o, precision)
    # the hydrogen update uses the H I rates only
    x_ref, _ = oracle.chem(g["n_H"], g["x_HI"], g["x_HII"], o["kph"], 1e13, 10, synth.ALPHA_B)
    grid.chem(1e13, 10, synth.ALPHA_B)
    np.testing.assert_allclose(grid.rates()["x_HI"], x_ref, rtol=parity.TOL[precision], atol=1e-12)
    grid.close()


def test_typed_grids_in_a_batch_and_with_finite_light():
    g, he, types = _typed(N=24, nsrc=9, seed=43)
    # in a batch beside an untyped grid
    batch = native.Batch(parity.ctx())
    typed = _grid(g, he, types, "fp32_mixed")
    plain = native.Grid(parity.ctx(), synth.clumpy(N=16, nsrc=3, seed=2), "fp32_mixed")
    s1 = batch.add(typed)
    batch.add(plain)
    batch.trace(checksums=True, **synth.DEFAULT_PARAMS)
    _compare(g, batch.budget(s1), typed, _oracle(g, he, types), "fp32_mixed")
    batch.close()
    typed.close()
    plain.close()
    # finite speed of light: three steps, each against the oracle's step
    dx = g["box_len_cm"] / 24
    grid = _grid(g, he, types, "fp64")
    fl = oracle.Flight()
    for step in range(3):
        b = grid.trace(checksums=True, light_cm=6.0 * dx, **synth.DEFAULT_PARAMS)
        o = _oracle(g, he, types, flight=fl, light_cm=6.0 * dx)
        assert b["n_halted"] == o["n_halted"] and b["n_resumed"] == (0 if step == 0 else prev)
        prev = b["n_halted"]
        np.testing.assert_array_equal(b["counts"], o["counts"])
        np.testing.assert_array_equal(b["hashes"], o["hashes"])
        assert b["segments"] == o["segments"]
        for t in range(3):
            ref = o["kph_types"][t]
            got = grid.rates_typed(t)["kph"]
            m = ref > 1e-8 * ref.max()
            np.testing.assert_allclose(got[m], ref[m], rtol=1e-6)
    grid.close()


def test_type_api_edges():
    g, he, types = _typed(N=12, nsrc=3, seed=47)
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    grid.set_source_types(types)
    with pytest.raises(native.RtError):
        grid.trace(**synth.DEFAULT_PARAMS)  # helium types without helium absorbers
    with pytest.raises(native.RtError):
        grid.rates_typed(1)
    with pytest.raises(native.RtError):
        grid.set_source_types([0, 1])  # wrong count
    with pytest.raises(native.RtError):
        grid.set_source_types([2, 2, 2])  # 15.6 eV is below the He II threshold
    bad = he[1].copy()
    bad[5] = -1.0
    with pytest.raises(native.RtError):
        grid.set_absorbers(he[0], bad)
    grid.set_absorbers(he[0], he[1])
    b = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    _compare(g, b, grid, _oracle(g, he, types), "fp32_mixed")
    grid.close()
