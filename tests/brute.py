"""Brute-force references used to pin the oracle.

Nothing here imports the oracle or the CUDA library.  Each helper computes a
quantity from first principles in a different way from the oracle, so that a
mistake in the oracle (a wrong sign, index or dropped term) shows up as a
mismatch:

* ``slab_segments`` intersects a ray with EVERY cell of a tiny grid (slab
  method) instead of walking the grid cell by cell;
* ``ring_layout`` is the closed-form HEALPix ring description (z and phi of
  each ring, Gorski et al. 2005) instead of the nested face algebra;
* ``split_tree`` enumerates the HEALPix packages that adaptive ray tracing
  creates in a transparent medium from the sorted list of every plane
  crossing of each ray, instead of a DDA;
* chemistry closed forms and exact equilibrium roots.
"""
from __future__ import annotations

from decimal import Decimal, getcontext

import numpy as np


def slab_segments(dims, s, n, r0=0.0):
    """Cells (k,3) crossed by the ray s + r n, r >= r0, with positive length, sorted by entry.

    Returns (cells, entry, exit) with cell units (cell width 1).
    """
    nx, ny, nz = dims
    s = np.asarray(s, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lo = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(np.float64)
    hi = lo + 1.0
    tin = np.full(lo.shape[0], r0)
    tout = np.full(lo.shape[0], np.inf)
    for a in range(3):
        if n[a] == 0.0:
            inside = (s[a] >= lo[:, a]) & (s[a] <= hi[:, a])
            tout = np.where(inside, tout, -np.inf)
            continue
        t1 = (lo[:, a] - s[a]) / n[a]
        t2 = (hi[:, a] - s[a]) / n[a]
        tin = np.maximum(tin, np.minimum(t1, t2))
        tout = np.minimum(tout, np.maximum(t1, t2))
    keep = tout > tin
    order = np.argsort(tin[keep], kind="stable")
    return lo[keep][order].astype(np.int64), tin[keep][order], tout[keep][order]


def box_exit(dims, s, n):
    """Distance from s along n to the boundary of the box [0, dims]."""
    t = np.inf
    for a in range(3):
        if n[a] > 0:
            t = min(t, (dims[a] - s[a]) / n[a])
        elif n[a] < 0:
            t = min(t, (0.0 - s[a]) / n[a])
    return t


def ring_layout(level: int):
    """Closed-form HEALPix rings at Nside = 2^level: list of (z, sorted phi array)."""
    N = 2 ** level
    rings = []
    for i in range(1, 4 * N):
        if i < N:
            z = 1.0 - i * i / (3.0 * N * N)
            phi = (np.pi / (2.0 * i)) * (np.arange(1, 4 * i + 1) - 0.5)
        elif i <= 3 * N:
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * N)
            sft = (i - N + 1) % 2
            phi = (np.pi / (2.0 * N)) * (np.arange(1, 4 * N + 1) - sft / 2.0)
        else:
            ii = 4 * N - i
            z = -(1.0 - ii * ii / (3.0 * N * N))
            phi = (np.pi / (2.0 * ii)) * (np.arange(1, 4 * ii + 1) - 0.5)
        rings.append((z, np.sort(np.mod(phi, 2 * np.pi))))
    return rings


def plane_crossings(dims, s, n):
    """Sorted distinct distances at which the ray crosses any integer plane inside the box."""
    ts = []
    for a in range(3):
        if n[a] == 0.0:
            continue
        b = np.arange(0, dims[a] + 1, dtype=np.float64)
        t = (b - s[a]) / n[a]
        ts.append(t[t > 0])
    if not ts:
        return np.array([])
    return np.unique(np.concatenate(ts))


def split_tree(dims, s, pix2vec, level0, phi_c, max_level):
    """Packages (level, pixel) created in a transparent medium.

    A package starting at radius r0 walks the cells between consecutive plane
    crossings beyond r0; it splits in the first cell, still inside the box,
    whose exit radius exceeds R_split(l) = sqrt(12 4^l / (4 pi Phi_c)), and
    its four children start at that cell's entry radius.
    """
    dims = np.asarray(dims)
    created = {l: set() for l in range(max_level + 1)}
    todo = [(level0, p, 0.0) for p in range(12 * 4 ** level0)]
    for (l, p, _) in todo:
        created[l].add(p)
    while todo:
        l, p, r0 = todo.pop()
        n = pix2vec(l, p)
        xs = plane_crossings(dims, s, n)
        exits = xs[xs > r0]
        rsplit = np.sqrt(12.0 * 4.0 ** l / (4.0 * np.pi * phi_c))
        entry = r0
        for e in exits:
            mid = s + 0.5 * (entry + e) * n
            if np.any(mid < 0) or np.any(mid > dims):
                break
            if l < max_level and e > rsplit:
                for k in range(4):
                    created[l + 1].add(4 * p + k)
                    todo.append((l + 1, 4 * p + k, entry))
                break
            entry = e
    return created


def equilibrium_x(alpha_n: float, k: float) -> Decimal:
    """Root x in [0,1] of alpha n (1-x)^2 = k x, in 50-digit decimal arithmetic."""
    getcontext().prec = 50
    a = Decimal(alpha_n)
    kk = Decimal(k)
    # a x^2 - (2a + k) x + a = 0, smaller root
    B = 2 * a + kk
    disc = B * B - 4 * a * a
    return (B - disc.sqrt()) / (2 * a)


def recombination_only_z(z0: float, alpha_n: float, t: float) -> float:
    """x_HII(t) for k = 0: dz/dt = -alpha n z^2."""
    return z0 / (1.0 + alpha_n * z0 * t)


def riccati_z(z0: float, alpha_n: float, k: float, t: float) -> float:
    """x_HII(t) for constant k: dz/dt = -alpha n z^2 + k (1 - z)."""
    a = alpha_n
    disc = np.sqrt(k * k + 4 * a * k)
    zp = (-k + disc) / (2 * a)  # stable equilibrium
    zm = (-k - disc) / (2 * a)
    lam = a * (zp - zm)
    e = np.exp(-lam * t)
    c = (z0 - zp) / (z0 - zm)
    return (zp - zm * c * e) / (1.0 - c * e)
