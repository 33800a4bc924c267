"""Adaptive radiative-transfer timestep (Sec. 3.4, Eqs. "dtelec", "dtchange").

TEST INFRASTRUCTURE ONLY (part of the oracle package; see its docstring).

Plain FP64 numpy, following the paper's steps in order:

1. per cell, Eq. "dtelec": dt_cell = eps_ion / |k_ph + n_e (C_H + alpha_B)|
   with C_H = 0 and n_e = n_H (1 - x_HI) (hydrogen only), in the cells
   "within the ionisation front", i.e. whose optical depth
   sigma_front n_HI dx exceeds tau_front (0.5 in the paper); every other
   cell takes dt_max (the paper's hydrodynamical timestep), and no cell more
   than dt_max;
2. smooth dt_cell with a Gaussian filter over the 3^3 cube around each cell;
3. dt_P = the minimum of the smoothed field;
4. Eq. "dtchange": dt_P = min(2 dt_prev, dt_P) when a previous step exists.

Readings (where the paper is silent): the filter's width is one cell,
weights exp(-|d|^2 / 2) for the 27 offsets d, renormalised over the
neighbours that lie inside the grid; tau is the cell's own optical depth
for the cross section sigma_front.
"""
from __future__ import annotations

import itertools

import numpy as np


def cell_timestep(n_H, x_HI, kph, dx_cm, eps_ion, alpha_B, sigma_front, tau_front, dt_max):
    """Step 1: per-cell timestep (flat arrays, FP64)."""
    n_H = np.asarray(n_H, dtype=np.float64)
    x = np.asarray(x_HI, dtype=np.float64)
    k = np.asarray(kph, dtype=np.float64)
    n_e = n_H * (1.0 - x)
    rate = np.abs(k + n_e * alpha_B)
    with np.errstate(divide="ignore"):
        dt = np.where(rate > 0, eps_ion / np.where(rate > 0, rate, 1.0), np.inf)
    front = (sigma_front * dx_cm) * n_H * x > tau_front
    return np.minimum(np.where(front, dt, dt_max), dt_max)


def smooth(field, dims):
    """Step 2: renormalised 3^3 Gaussian filter (x fastest: index i + nx(j + ny k))."""
    nx, ny, nz = dims
    f = np.asarray(field, dtype=np.float64).reshape(nz, ny, nx)
    acc = np.zeros_like(f)
    wsum = np.zeros_like(f)
    for dz, dy, dxo in itertools.product((-1, 0, 1), repeat=3):
        w = np.exp(-(dxo * dxo + dy * dy + dz * dz) / 2.0)
        # neighbour (k + dz, j + dy, i + dxo) of every cell whose neighbour is inside
        src = f[max(dz, 0):nz + min(dz, 0), max(dy, 0):ny + min(dy, 0), max(dxo, 0):nx + min(dxo, 0)]
        sl = (slice(max(-dz, 0), nz + min(-dz, 0)), slice(max(-dy, 0), ny + min(-dy, 0)),
              slice(max(-dxo, 0), nx + min(-dxo, 0)))
        acc[sl] += w * src
        wsum[sl] += w
    return (acc / wsum).reshape(-1)


def rt_timestep(dims, dx_cm, n_H, x_HI, kph, *, eps_ion=0.05, alpha_B=2.59e-13, sigma_front=6.3e-18,
                tau_front=0.5, dt_max=np.inf, dt_prev=0.0):
    """Steps 1-4: the radiative-transfer timestep dt_P (seconds)."""
    dtc = cell_timestep(n_H, x_HI, kph, dx_cm, eps_ion, alpha_B, sigma_front, tau_front, dt_max)
    dt = float(np.min(smooth(dtc, dims)))
    if dt_prev > 0:
        dt = min(2.0 * dt_prev, dt)
    return dt
