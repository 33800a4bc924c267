"""Pins for the oracle's adaptive RT timestep (Sec. 3.4, Eqs. "dtelec", "dtchange").

Checked against: the closed form in a uniform ionisation front (smoothing a
constant is the identity); the smoothing done independently with
scipy.ndimage.correlate (Gaussian weights, zero padding, renormalised by the
correlation of the grid's indicator); the selection of front cells by their
optical depth; and the factor-of-two cap on the growth of dt_P.
"""
import numpy as np
import pytest

from oracle import timestep

ALPHA = 2.59e-13


def _state(dims, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    n_H = 10 ** rng.uniform(-3, -1, n)
    x = rng.uniform(0, 1, n)
    k = 10 ** rng.uniform(-16, -11, n)
    return n_H, x, k


def test_uniform_front_is_the_closed_form():
    dims = (6, 5, 4)
    n = 6 * 5 * 4
    n_H, x, k = np.full(n, 0.1), np.full(n, 0.7), np.full(n, 3e-13)
    dt = timestep.rt_timestep(dims, 1e21, n_H, x, k, eps_ion=0.05, alpha_B=ALPHA, dt_max=1e20)
    assert dt == pytest.approx(0.05 / (3e-13 + 0.1 * 0.3 * ALPHA), rel=1e-13)


@pytest.mark.parametrize("dims", [(7, 6, 5), (1, 4, 9), (3, 1, 1)])
def test_smoothing_matches_scipy(dims):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(sum(dims))
    f = rng.uniform(0.5, 2.0, int(np.prod(dims)))
    w = np.exp(-np.add.outer(np.add.outer(np.arange(-1, 2) ** 2, np.arange(-1, 2) ** 2),
                             np.arange(-1, 2) ** 2) / 2.0)
    F = f.reshape(dims[2], dims[1], dims[0])
    num = ndimage.correlate(F, w, mode="constant", cval=0.0)
    den = ndimage.correlate(np.ones_like(F), w, mode="constant", cval=0.0)
    np.testing.assert_allclose(timestep.smooth(f, dims), (num / den).reshape(-1), rtol=1e-14)


def test_only_front_cells_limit_the_step():
    dims = (8, 8, 8)
    n_H, x, k = _state(dims, 3)
    dx = 3.0e20
    tau = 6.3e-18 * n_H * x * dx
    dtc = timestep.cell_timestep(n_H, x, k, dx, 0.05, ALPHA, 6.3e-18, 0.5, 1e15)
    assert np.all(dtc[tau <= 0.5] == 1e15)
    m = tau > 0.5
    np.testing.assert_allclose(dtc[m], np.minimum(1e15, 0.05 / (k[m] + n_H[m] * (1 - x[m]) * ALPHA)), rtol=1e-15)
    # a fully ionised grid has no front: dt_P = dt_max
    assert timestep.rt_timestep(dims, dx, n_H, np.full(512, 1e-6), k, dt_max=1e15) == pytest.approx(1e15, rel=1e-14)


def test_growth_is_capped_at_twice_the_previous_step():
    dims = (4, 4, 4)
    n_H, x, k = _state(dims, 5)
    free = timestep.rt_timestep(dims, 3e20, n_H, x, k, dt_max=1e16)
    assert timestep.rt_timestep(dims, 3e20, n_H, x, k, dt_max=1e16, dt_prev=0.25 * free) == 0.5 * free
    assert timestep.rt_timestep(dims, 3e20, n_H, x, k, dt_max=1e16, dt_prev=free) == free
