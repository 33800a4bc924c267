"""Pins for the oracle's HEALPix nested scheme (Sec. 2.1; Step 3a).

What fixes the answer: N_pix = 12 * 4^l equal-area pixels (Sec. 2.1), nested
children p' = 4p + {0,1,2,3} (Sec. 2.1), and the closed-form ring layout of
HEALPix (Gorski et al. 2005): ring z values and equally spaced azimuths.
"""
import numpy as np
import pytest

import brute
import oracle


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_pixel_count_unit_norm_distinct(level):
    npix = 12 * 4 ** level
    v = oracle.pix2vec(level, np.arange(npix))
    assert v.shape == (npix, 3)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=2e-16 * 8)
    # all distinct and the mean vanishes (the pixelisation is symmetric)
    assert len({tuple(np.round(x, 12)) for x in v}) == npix
    np.testing.assert_allclose(v.sum(axis=0), 0.0, atol=1e-12)


def test_base_layout():
    z, phi = oracle.pix2ang(0, np.arange(12))
    np.testing.assert_array_equal(z[:4], 2.0 / 3.0)
    np.testing.assert_array_equal(z[4:8], 0.0)
    np.testing.assert_array_equal(z[8:], -2.0 / 3.0)
    np.testing.assert_allclose(phi[:4], (2 * np.arange(4) + 1) * np.pi / 4, rtol=1e-15)
    np.testing.assert_allclose(phi[4:8], np.arange(4) * np.pi / 2, rtol=1e-15)
    np.testing.assert_allclose(phi[8:], (2 * np.arange(4) + 1) * np.pi / 4, rtol=1e-15)


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_ring_layout_closed_form(level):
    npix = 12 * 4 ** level
    z, phi = oracle.pix2ang(level, np.arange(npix))
    rings = brute.ring_layout(level)
    assert sum(len(p) for _, p in rings) == npix
    used = np.zeros(npix, dtype=bool)
    for zr, phis in rings:
        sel = np.abs(z - zr) < 1e-14
        assert sel.sum() == len(phis), (zr, sel.sum(), len(phis))
        np.testing.assert_allclose(np.sort(phi[sel]), phis, atol=1e-13)
        used |= sel
    assert used.all()


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_children_are_nested(level):
    npix = 12 * 4 ** level
    child = np.arange(4 * npix)
    zc, pc = oracle.pix2ang(level + 1, child)
    parent = oracle.ang2pix(level, zc, pc)
    np.testing.assert_array_equal(parent, child // 4)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_round_trip(level):
    npix = 12 * 4 ** level
    p = np.arange(npix)
    z, phi = oracle.pix2ang(level, p)
    np.testing.assert_array_equal(oracle.ang2pix(level, z, phi), p)
    v = oracle.pix2vec(level, p)
    np.testing.assert_allclose(v[:, 2], z, rtol=0, atol=0)
    np.testing.assert_allclose(np.arctan2(v[:, 1], v[:, 0]) % (2 * np.pi), phi, atol=1e-13)


def test_equal_area():
    """Uniform directions fall into the 192 level-2 pixels with equal probability."""
    rng = np.random.default_rng(7)
    m = 120000
    z = rng.uniform(-1, 1, m)
    phi = rng.uniform(0, 2 * np.pi, m)
    p = oracle.ang2pix(2, z, phi)
    h = np.bincount(p.astype(np.int64), minlength=192)
    assert h.size == 192
    expect = m / 192
    chi2 = np.sum((h - expect) ** 2 / expect)
    # 191 degrees of freedom: mean 191, sd 19.5; a wrong partition gives >> 1000
    assert chi2 < 300, chi2


def test_exact_zero_and_mirror_components():
    """Vanishing components are exact zeros; pixels at 45 degrees have |n_x| == |n_y| exactly."""
    for level in range(0, 6):
        npix = 12 * 4 ** level
        v = oracle.pix2vec(level, np.arange(npix))
        z, phi = oracle.pix2ang(level, np.arange(npix))
        q = phi / (np.pi / 2)
        on_axis = np.abs(q - np.round(q)) < 1e-12
        assert np.all((v[on_axis, 0] == 0) | (v[on_axis, 1] == 0))
        diag = np.abs(q - np.floor(q) - 0.5) < 1e-12
        assert np.all(np.abs(v[diag, 0]) == np.abs(v[diag, 1]))
        eq = np.abs(z) < 1e-15
        assert np.all(v[eq, 2] == 0)
