"""Pins for photon types in the oracle (Sec. 3.2: mono-chromatic packages of
a photon type, absorbed by that type's species; reading R16).

* a He I-type source in a medium whose n_HeI equals another medium's n_HI,
  with the same excess energy E - E_i, reproduces the H I-type trace exactly;
* types do not interact: each type's rates equal the trace of that type's
  sources alone, and the photon budgets add;
* a type whose absorber is absent crosses the box unabsorbed, and its
  k_ph per absorber is the optically thin limit sigma P dr / V (reading R5);
* Gamma / k_ph = (E - E_i) per type, E_i = 13.6, 24.6, 54.4 eV.
"""
import numpy as np
import pytest

import oracle
from paper_1012_2865_gb300 import synth

EV = 1.602176634e-12
E_ION = (13.6, 24.6, 54.4)


def _trace(g, **kw):
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], **kw)


def _he_medium(g, seed=3):
    """n_HeI, n_HeII: a different clumpy pattern from the hydrogen's."""
    n = g["n_H"].size
    rng = np.random.default_rng(seed)
    he1 = synth.round_f32(0.08 * g["n_H"] * rng.uniform(0.2, 1.0, n))
    he2 = synth.round_f32(0.02 * g["n_H"] * rng.uniform(0.0, 1.0, n))
    return np.stack([he1, he2])


def test_relabelled_species_reproduce_the_hydrogen_trace():
    g = synth.clumpy(N=20, nsrc=5, seed=17)
    g["x_HI"] = np.full(g["n_H"].size, 0.3)
    h = _trace(g)
    n_hi = g["n_H"] * g["x_HI"]
    he = dict(g, e_ph_eV=g["e_ph_eV"] + (E_ION[1] - E_ION[0]))
    r = _trace(he, src_type=np.ones(5, dtype=int), n_he=np.stack([n_hi, np.zeros_like(n_hi)]))
    np.testing.assert_array_equal(r["kph_types"][1], h["kph"])
    # E - E_i agree to rounding ((E + 11) - 24.6 vs E - 13.6)
    np.testing.assert_allclose(r["gamma_types"][1], h["gamma"], rtol=1e-14, atol=0)
    assert np.all(r["kph_types"][0] == 0) and np.all(r["kph_types"][2] == 0)
    for key in ("counts", "hashes", "budget"):
        np.testing.assert_array_equal(r[key], h[key])
    assert r["segments"] == h["segments"]


def test_types_do_not_interact():
    g = synth.clumpy(N=20, nsrc=9, seed=23)
    g["x_HI"] = np.full(g["n_H"].size, 0.05)
    he = _he_medium(g)
    types = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2])
    g["e_ph_eV"] = np.array([E_ION[t] + 6.0 + k for k, t in enumerate(types)])
    r = _trace(g, src_type=types, n_he=he)
    em = 0.0
    for t in range(3):
        sel = types == t
        gt = dict(g, pos_cm=g["pos_cm"][sel], ndot=g["ndot"][sel], e_ph_eV=g["e_ph_eV"][sel],
                  sigma_cm2=g["sigma_cm2"][sel])
        rt = _trace(gt, src_type=types[sel], n_he=he)
        np.testing.assert_array_equal(r["kph_types"][t], rt["kph_types"][t])
        np.testing.assert_array_equal(r["gamma_types"][t], rt["gamma_types"][t])
        for u in range(3):
            if u != t:
                assert np.all(rt["kph_types"][u] == 0)
        em += rt["budget"][0]
        assert abs(rt["budget"][0] - rt["budget"][1] - rt["budget"][2]) <= 1e-12 * rt["budget"][0]
    assert abs(r["budget"][0] - em) <= 1e-12 * em
    assert r["kph_types"][1].max() > 0 and r["kph_types"][2].max() > 0


def test_type_without_absorber_is_unabsorbed():
    """He II photons in a medium without He II: every photon escapes; the rate
    per absorber is the thin limit.  He I photons in the same box are absorbed."""
    N = 12
    g = synth.clumpy(N=N, nsrc=2, seed=5)
    he = _he_medium(g)
    he[1] = 0.0
    g["e_ph_eV"] = np.array([60.0, 30.0])
    r = _trace(g, src_type=[2, 1], n_he=he, level0=1)
    b2 = _trace(dict(g, pos_cm=g["pos_cm"][:1], ndot=g["ndot"][:1], e_ph_eV=g["e_ph_eV"][:1],
                     sigma_cm2=g["sigma_cm2"][:1]), src_type=[2], n_he=he)
    assert b2["budget"][1] == 0.0 and b2["budget"][2] == b2["budget"][0]
    # thin limit: sum over cells of k V / sigma = sum over segments of P dr (photons/s x cm)
    dx = g["box_len_cm"] / N
    path = np.sum(b2["kph_types"][2]) * dx ** 3 / g["sigma_cm2"][0]
    assert path > 0
    assert r["budget"][1] > 0  # the He I source is absorbed
    # every photon of the He II source travels from the source to the box edge: the
    # photon-weighted path is between the nearest and the farthest face distances
    s = g["pos_cm"][0]
    near = min(np.min(s), np.min(N * dx - s))
    far = np.sqrt(np.sum(np.maximum(s, N * dx - s) ** 2))
    assert near * g["ndot"][0] <= path <= far * g["ndot"][0]


@pytest.mark.parametrize("t", [0, 1, 2])
def test_heating_per_type(t):
    g = synth.clumpy(N=12, nsrc=1, seed=29)
    he = _he_medium(g)
    g["e_ph_eV"] = np.array([E_ION[t] + 7.5])
    r = _trace(g, src_type=[t], n_he=he)
    k, gm = r["kph_types"][t], r["gamma_types"][t]
    m = k > 0
    np.testing.assert_allclose(gm[m] / k[m], 7.5 * EV, rtol=1e-14)


def test_he_types_need_their_absorbers():
    g = synth.clumpy(N=8, nsrc=1, seed=1)
    with pytest.raises(ValueError):
        _trace(g, src_type=[1])
