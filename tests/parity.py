"""Shared helpers for GPU-vs-oracle parity tests.

Tolerances (stated by the method's target and written here once):
* packages created per HEALPix level and the checksum of the created
  (source, level, pixel) set: bit-exact, both paths;
* k_ph and Gamma: relative 1e-6 (FP64 path) / 1e-3 (FP32-mixed path) in every
  cell that receives more than 1e-8 of the emitted photons, where the photons
  a cell receives are measured by the photon path length through it,
  k_ph V / (sigma dx) (photons/s times cell lengths);
* photon budget: emitted = absorbed + escaped to 1e-12 relative on the GPU,
  and each term within 1e-9 (FP64) / 1e-5 (FP32) of the emitted rate from
  the oracle's;
* x_HI after the implicit update: relative 1e-6 (FP64) / 1e-3 (FP32) plus
  an absolute 1e-12.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1012_2865_gb300 import native, synth

TOL = {"fp64": 1e-6, "fp32_mixed": 1e-3}
BUDGET_TOL = {"fp64": 1e-9, "fp32_mixed": 1e-5}

_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        _ctx = native.rt_ctx_create(0)
    return _ctx


def run_oracle(g, **params):
    p = dict(synth.DEFAULT_PARAMS)
    p.update(params)
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"],
                        g["e_ph_eV"], g["sigma_cm2"], **p)


def run_gpu(g, precision="fp64", **params):
    p = dict(synth.DEFAULT_PARAMS, checksums=True)
    p.update(params)
    grid = native.Grid(ctx(), g, precision)
    b = grid.trace(**p)
    r = grid.rates()
    return grid, b, r


def receiving_mask(g, kph, emitted):
    """Cells receiving more than 1e-8 of the emitted photons (path-length measure)."""
    dx = g["box_len_cm"] / g["dims"][0]
    sigma = float(np.max(g["sigma_cm2"])) if len(g["sigma_cm2"]) else 1.0
    recv = kph * dx ** 3 / (sigma * dx)
    return recv > 1e-8 * emitted


def assert_trace_parity(g, b, r, o, precision="fp64", exact_segments=None):
    tol = TOL[precision]
    assert b["status"] == 0
    np.testing.assert_array_equal(b["counts"], o["counts"], err_msg="packages per level")
    np.testing.assert_array_equal(b["hashes"], o["hashes"], err_msg="created-set checksum")
    if exact_segments is None:
        exact_segments = precision == "fp64"
    if exact_segments:
        assert b["segments"] == o["segments"], (b["segments"], o["segments"])
    em = o["budget"][0]
    if em > 0:
        assert abs(b["emitted"] - b["absorbed"] - b["escaped"]) <= 1e-12 * b["emitted"]
        bt = BUDGET_TOL[precision]
        assert abs(b["emitted"] - em) <= bt * em
        assert abs(b["absorbed"] - o["budget"][1]) <= bt * em
        assert abs(b["escaped"] - o["budget"][2]) <= bt * em
    mask = receiving_mask(g, o["kph"], em)
    worst = {}
    for key in ("kph", "gamma"):
        ref = o[key][mask]
        got = np.asarray(r[key], dtype=np.float64)[mask]
        nz = ref != 0
        if nz.any():
            rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
            assert rel.max() <= tol, (key, float(rel.max()), int(np.argmax(rel)))
            worst[key] = float(rel.max())
        assert np.all(got[~nz] == 0) or np.max(np.abs(got[~nz])) <= tol * max(np.abs(ref).max(), 1e-300)
    return worst
