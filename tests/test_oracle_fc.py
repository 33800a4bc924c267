"""Pins for the optional covering-factor correction f_c (Sec. 2.3, Eq. "fc").

f_c scales each segment's k_ph and Gamma contribution by
(1/2 + D_edge/L_pix)^2 (capped at 1), where L_pix = r theta_pix is the width of
the (square) pixel where the segment starts and D_edge the distance from the
segment's midpoint to the nearest cell face along the axes.  It leaves dP
untouched, so every decision and the photon budget are those of the
uncorrected trace.  Checked here: those invariants; two worked cases where a
level-0 ray runs along +x through a one-cell-thick row of cells, so that the
geometry fixes D_edge and the per-cell ratio k_fc/k is (1/2 + D_edge/L_pix)^2;
and the paper's observation that the correction makes the optically thin
field more spherical at Phi_c = 5.1 (Sec. 8, "Improvements from the covering
factor correction").
"""
import numpy as np
import pytest

import oracle
from paper_1012_2865_gb300 import synth


def _trace(g, **kw):
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], **kw)


def test_fc_changes_only_the_rates():
    g = synth.clumpy(N=24, nsrc=6, seed=9)
    a = _trace(g)
    b = _trace(g, fc=True)
    for key in ("counts", "hashes"):
        np.testing.assert_array_equal(a[key], b[key])
    assert a["segments"] == b["segments"]
    np.testing.assert_array_equal(a["budget"], b["budget"])
    m = a["kph"] > 0
    ratio = b["kph"][m] / a["kph"][m]
    assert ratio.min() >= 0.25 - 1e-12 and ratio.max() <= 1.0 + 1e-12
    assert ratio.min() < 0.9  # the correction is active somewhere
    assert np.all(b["kph"][~m] == 0)
    mg = a["gamma"] > 0
    rg = b["gamma"][mg] / a["gamma"][mg]
    assert rg.min() >= 0.25 - 1e-12 and rg.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("y_off", [0.0, 0.2])
def test_fc_on_a_ray_along_x(y_off):
    """Source in cell 0 of an 8 x 1 x 1 row at height 0.5 - y_off; the level-0
    pixel (z = 0, phi = 0) is exactly +x (pixel directions keep exact zeros).
    Segment k >= 1 starts at r = k - 0.5 (cell widths) and ends at k + 0.5, so
    its midpoint sits on the cell's centre plane in x and z and y_off below it
    in y: D_edge = 1/2 - y_off.  Only this ray reaches cells 1..7 (the others
    leave the one-cell-thick row in cell 0), and Phi_c is so small that
    nothing splits."""
    N = 8
    box = synth.box_cm(N)
    dx = box / N
    g = dict(dims=np.array([N, 1, 1]), box_len_cm=box, n_H=np.full(N, 1e-6), x_HI=np.full(N, 1.0),
             pos_cm=np.array([[0.5 * dx, (0.5 - y_off) * dx, 0.5 * dx]]), ndot=np.array([1e48]),
             e_ph_eV=np.array([20.0]), sigma_cm2=np.array([synth.SIGMA_HI]))
    a = _trace(g, level0=0, phi_c=1e-9)
    b = _trace(g, level0=0, phi_c=1e-9, fc=True)
    theta0 = np.sqrt(4 * np.pi / 12)  # width of a level-0 pixel taken as a square
    k = np.arange(1, N)
    L = (k - 0.5) * theta0
    expect = np.minimum(1.0, (0.5 + (0.5 - y_off) / L) ** 2)
    np.testing.assert_allclose(b["kph"][1:] / a["kph"][1:], expect, rtol=1e-12)
    assert b["kph"][0] == a["kph"][0]  # every segment in cell 0 starts at r = 0: f_c = 1


def _thin_dev(fc, phi_c=5.1, N=32, src=(15, 16, 14)):
    g = synth.stromgren(N)
    g["n_H"] = synth.round_f32(np.full(N ** 3, 1e-3))
    g["x_HI"] = np.full(N ** 3, 1e-8)
    dx = g["box_len_cm"] / N
    g["pos_cm"] = synth.cell_centre_cm(np.array([src]), dx)
    r = _trace(g, phi_c=phi_c, fc=fc)
    i = np.arange(N) + 0.5
    X = (i[None, None, :] - (src[0] + 0.5)) ** 2 + (i[None, :, None] - (src[1] + 0.5)) ** 2 + \
        (i[:, None, None] - (src[2] + 0.5)) ** 2
    rc = np.sqrt(X).reshape(-1)
    sel = (rc > 3) & (rc < N / 2 - 2)
    k_thin = g["sigma_cm2"][0] * g["ndot"][0] / (4 * np.pi * (rc[sel] * dx) ** 2)
    return r["kph"][sel] / k_thin


def test_fc_makes_the_thin_field_more_spherical():
    """Optically thin medium, Phi_c = 5.1 (the setting of the paper's test):
    the relative scatter of k_ph r^2 about its mean is smaller with f_c."""
    a = _thin_dev(False)
    b = _thin_dev(True)
    assert np.std(b) / np.mean(b) < np.std(a) / np.mean(a)
    assert 0.7 < np.mean(b) / np.mean(a) < 1.0  # f_c only removes contributions
