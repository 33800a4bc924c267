"""Pins for the oracle's hydrogen-only ionisation update (Eq. "dndt", Step 6).

Reading: backward Euler on dx/dt = alpha_B n_H (1 - x)^2 - k x with nsub equal
substeps and k frozen over the step.  Pinned against the implicit equation
itself, the exact equilibrium root, and the closed-form solutions for k = 0
(pure recombination) and constant k (a Riccati equation).
"""
from decimal import Decimal

import numpy as np
import pytest

import brute
import oracle

ALPHA = 2.59e-13


def _one(n, x, k, dt, nsub):
    xs, zs = oracle.chem(np.array([n]), np.array([x]), np.array([1.0 - x]), np.array([k]), dt, nsub,
                         ALPHA)
    return xs[0], zs[0]


@pytest.mark.parametrize("n,x,k,h", [(1e-3, 1.0, 1e-12, 3e13), (1e-2, 0.3, 5e-11, 1e14),
                                     (1.0, 1e-6, 1e-9, 1e10), (1e-3, 0.999, 0.0, 1e15)])
def test_backward_euler_residual(n, x, k, h):
    """One substep solves x' = x + h (alpha n (1 - x')^2 - k x') to rounding."""
    x1, z1 = _one(n, x, k, h, 1)
    assert x1 + z1 == pytest.approx(1.0, abs=2e-16)
    lhs = x1 - x
    rhs = h * (ALPHA * n * z1 * z1 - k * x1)
    scale = max(abs(x1), abs(x), abs(h * ALPHA * n), abs(h * k * x1))
    assert abs(lhs - rhs) <= 1e-14 * scale


@pytest.mark.parametrize("n,k", [(1e-3, 1e-12), (1e-3, 1e-9), (1e-2, 1e-14), (3e-4, 5e-8)])
def test_fixed_point_is_equilibrium(n, k):
    """A long step lands on the root of alpha n (1-x)^2 = k x (exact decimal root)."""
    x, z = _one(n, 0.5, k, 1e20, 4)
    xe = brute.equilibrium_x(ALPHA * n, k)
    assert abs(Decimal(x) - xe) <= Decimal(1e-13) * xe
    assert abs(Decimal(z) - (1 - xe)) <= Decimal(1e-13)


def test_small_neutral_fraction_keeps_relative_accuracy():
    """x_HI ~ 1e-10 deep inside an HII region keeps ~14 digits (complementary pair)."""
    n, k = 1e-3, 1e-4
    x, _ = _one(n, 0.5, k, 1e18, 2)
    xe = brute.equilibrium_x(ALPHA * n, k)
    assert float(xe) < 1e-8
    assert abs(Decimal(x) - xe) <= Decimal(1e-13) * xe


def test_recombination_closed_form_first_order():
    """k = 0: x_HII(t) = z0 / (1 + alpha n z0 t); backward Euler converges at first order."""
    n, z0, t = 1e-3, 0.9, 3e15
    exact = brute.recombination_only_z(z0, ALPHA * n, t)
    errs = []
    for nsub in (50, 100, 200, 400):
        _, z = _one(n, 1.0 - z0, 0.0, t, nsub)
        errs.append(abs(z - exact))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(0.9 < r < 1.1 for r in rates), rates
    assert errs[-1] / exact < 2e-3


def test_constant_rate_riccati_closed_form():
    n, k, z0, t = 1e-3, 2e-13, 0.01, 6e13  # t ~ one relaxation time
    exact = brute.riccati_z(z0, ALPHA * n, k, t)
    _, z1 = _one(n, 1.0 - z0, k, t, 200)
    _, z2 = _one(n, 1.0 - z0, k, t, 400)
    assert abs(z2 - exact) < abs(z1 - exact)
    assert abs(z2 - exact) / exact < 2e-3
    assert abs(z1 - exact) / abs(z2 - exact) == pytest.approx(2.0, rel=0.1)
