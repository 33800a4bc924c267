"""Finite speed of light on the GPU (Sec. 2.1, Step 3j) against the oracle.

Every trace of a sequence is compared with the oracle's trace of the same
step, each side carrying its own packages in flight from step to step:
packages created per level and the created-set checksum bit-exact, the
segment count exact on the FP64 path, k_ph and Gamma within the parity
tolerances, the photon budget (emitted, absorbed, escaped, resumed, halted),
and the packages in flight as a set: the same (source, level, pixel, age,
cell) each, with radius, optical depth and photons equal to rounding.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

PREC = ["fp64", "fp32_mixed"]
P_TOL = {"fp64": 1e-12, "fp32_mixed": 2e-5}


def _static(N=24, nsrc=4, seed=21, x=0.02):
    g = synth.clumpy(N=N, nsrc=nsrc, seed=seed)
    g["x_HI"] = np.full(N ** 3, x)
    g["x_HII"] = 1.0 - g["x_HI"]
    return g


def _diag(g):
    return float(np.sqrt(np.sum(np.asarray(g["dims"], dtype=np.float64) ** 2)))


def _oracle(g, fl, light_cm, **kw):
    p = dict(synth.DEFAULT_PARAMS)
    p.update(kw)
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], flight=fl, light_cm=light_cm, **p)


def _compare_flight(g, got, ref, precision, tau_rtol=None):
    dx = g["box_len_cm"] / g["dims"][0]
    assert got.size == ref.size
    if got.size == 0:
        return
    a = got[np.lexsort((got["age"], got["pix"], got["level"], got["src"]))]
    b = ref[np.lexsort((ref["age"], ref["pix"], ref["level"], ref["src"]))]
    for k_got, k_ref in (("src", "src"), ("level", "level"), ("pix", "pix"), ("age", "age"), ("cell", "cell")):
        np.testing.assert_array_equal(a[k_got].astype(np.int64), b[k_ref].astype(np.int64), err_msg=k_got)
    np.testing.assert_allclose(a["r_cm"] / dx, b["r"], rtol=1e-15 if precision == "fp64" else 1e-12)
    if tau_rtol is None:
        tau_rtol = 1e-13 if precision == "fp64" else 1e-9
    np.testing.assert_allclose(a["tau"], b["tau"], rtol=tau_rtol, atol=1e-12)
    # P - P (1 - e^-tau) loses relative accuracy as e^-tau falls, on both
    # sides: the bound is relative to the unattenuated lineage, P e^tau
    err = np.abs(a["P"] - b["P"])
    assert np.all(err <= P_TOL[precision] * b["P"] + 1e-14 * b["P"] * np.exp(b["tau"])), \
        float(np.max(err / b["P"]))


def _compare_step(g, b, r, o, precision):
    assert b["status"] == 0
    np.testing.assert_array_equal(b["counts"], o["counts"], err_msg="packages per level")
    np.testing.assert_array_equal(b["hashes"], o["hashes"], err_msg="created-set checksum")
    if precision == "fp64":
        assert b["segments"] == o["segments"], (b["segments"], o["segments"])
    assert b["n_halted"] == o["n_halted"]
    total = o["budget"][0] + o["resumed"]
    bt = parity.BUDGET_TOL[precision]
    for got, ref in ((b["emitted"], o["budget"][0]), (b["absorbed"], o["budget"][1]), (b["escaped"], o["budget"][2]),
                     (b["resumed"], o["resumed"]), (b["halted"], o["halted"])):
        assert abs(got - ref) <= bt * total, (got, ref)
    lhs = b["emitted"] + b["resumed"]
    assert abs(lhs - b["absorbed"] - b["escaped"] - b["halted"]) <= 1e-12 * max(lhs, 1e-300)
    mask = parity.receiving_mask(g, o["kph"], total)
    for key in ("kph", "gamma"):
        ref = o[key][mask]
        got = np.asarray(r[key], dtype=np.float64)[mask]
        nz = ref != 0
        if nz.any():
            rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
            assert rel.max() <= parity.TOL[precision], (key, float(rel.max()))


@pytest.mark.parametrize("precision", PREC)
def test_static_medium_step_by_step(precision):
    g = _static()
    dx = g["box_len_cm"] / g["dims"][0]
    light = 3.7 * dx
    grid = native.Grid(parity.ctx(), g, precision)
    fl = oracle.Flight()
    M = int(np.ceil(_diag(g) / 3.7)) + 2
    for step in range(M):
        b = grid.trace(checksums=True, light_cm=light, **synth.DEFAULT_PARAMS)
        o = _oracle(g, fl, light)
        _compare_step(g, b, grid.rates(), o, precision)
        assert b["n_resumed"] == (0 if step == 0 else prev_halted)
        prev_halted = b["n_halted"]
        _compare_flight(g, grid.in_flight(), fl.packages, precision)
    # the last step is the steady state: the infinite-speed trace's packages
    inf = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    np.testing.assert_array_equal(b["counts"], inf["counts"])
    np.testing.assert_array_equal(b["hashes"], inf["hashes"])
    assert grid.in_flight().size == 0  # an infinite-speed trace drops what was in flight
    grid.close()


@pytest.mark.parametrize("precision", PREC)
def test_pulse_with_chemistry_and_rate_changes(precision):
    """Application 5 (Eq. "test12") on a small box: the rate changes every
    step, a level change in between, and the chemistry couples the steps."""
    N = 24
    g = synth.pulse(N)
    dx = g["box_len_cm"] / N
    light = 3.1 * dx
    dt = 0.2 * synth.MYR_S
    t0 = 10 * dt
    grid = native.Grid(parity.ctx(), g, precision)
    fl = oracle.Flight()
    x, z = g["x_HI"].copy(), g["x_HII"].copy()
    for step in range(9):
        g["ndot"] = np.array([float(synth.pulse_rate(step * dt, t0_s=t0))])
        grid.set_source_rates(g["ndot"])
        kw = dict(synth.DEFAULT_PARAMS)
        if step == 4:
            kw["level0"] = 2  # the unit of every source changes with packages in flight
        b = grid.trace(checksums=True, light_cm=light, **kw)
        go = dict(g, x_HI=x)
        o = _oracle(go, fl, light, **kw)
        _compare_step(go, b, grid.rates(), o, precision)
        # the media differ by the chemistry's response to the rates' rounding
        _compare_flight(g, grid.in_flight(), fl.packages, precision, tau_rtol=1e-9 if precision == "fp64" else 1e-4)
        grid.chem(dt, 10, synth.ALPHA_B)
        x, z = oracle.chem(g["n_H"], x, z, o["kph"], dt, 10, synth.ALPHA_B)
    grid.close()


@pytest.mark.parametrize("precision", PREC)
def test_dark_sources_and_passes(precision):
    """One emission, then dark steps, traced in three passes: the photons in
    flight are delivered exactly once, as in the oracle."""
    g = _static(seed=33, nsrc=5)
    dx = g["box_len_cm"] / g["dims"][0]
    light = 5.3 * dx
    grid = native.Grid(parity.ctx(), g, precision)
    fl = oracle.Flight()
    ndot = g["ndot"].copy()
    M = int(np.ceil(_diag(g) / 5.3)) + 2
    for step in range(M):
        g["ndot"] = ndot if step == 0 else np.zeros_like(ndot)
        grid.set_source_rates(g["ndot"])
        b = grid.trace(checksums=True, light_cm=light, passes=3, **synth.DEFAULT_PARAMS)
        assert b["passes"] == 3
        o = _oracle(g, fl, light)
        _compare_step(g, b, grid.rates(), o, precision)
        _compare_flight(g, grid.in_flight(), fl.packages, precision)
    assert b["halted"] == 0.0
    grid.close()


def test_store_of_halted_packages_grows():
    """More packages halt than a new store holds (2^16): the trace is redone
    with a larger store and matches the oracle."""
    N = 48
    g = synth.pulse(N)
    rng = np.random.default_rng(5)
    pos, ndot, e, sg = synth.random_sources((N, N, N), g["box_len_cm"] / N, 24, 1e52, 1e54, rng)
    g.update(pos_cm=pos, ndot=ndot, e_ph_eV=e, sigma_cm2=sg)
    dx = g["box_len_cm"] / N
    light = 6.5 * dx
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    fl = oracle.Flight()
    for step in range(2):
        b = grid.trace(checksums=True, light_cm=light, level0=2, phi_c=5.1, f_term=1e-10, max_level=14)
        o = _oracle(g, fl, light, level0=2)
        assert b["n_halted"] > (1 << 16)
        _compare_step(g, b, grid.rates(), o, "fp32_mixed")
        _compare_flight(g, grid.in_flight(), fl.packages, "fp32_mixed")
    grid.close()


def test_api_edges():
    ctx = parity.ctx()
    g = _static(N=16, nsrc=2)
    dx = g["box_len_cm"] / 16
    grid = native.Grid(ctx, g, "fp32_mixed")
    b = grid.trace(light_cm=2.5 * dx, **synth.DEFAULT_PARAMS)
    assert b["n_halted"] > 0 and grid.in_flight().size == b["n_halted"]
    with pytest.raises(native.RtError):
        grid.trace(light_cm=-1.0, **synth.DEFAULT_PARAMS)
    with pytest.raises(native.RtError):
        grid.set_source_rates(np.ones(3))
    assert grid.in_flight().size == b["n_halted"]  # rejected calls change nothing
    native.rt_clear_sources(grid.h)
    assert grid.in_flight().size == 0
    native.rt_add_sources(grid.h, g["pos_cm"], g["ndot"], g["e_ph_eV"], g["sigma_cm2"])
    b2 = grid.trace(light_cm=2.5 * dx, **synth.DEFAULT_PARAMS)
    assert b2["n_resumed"] == 0 and b2["resumed"] == 0.0
    batch = native.Batch(ctx)
    batch.add(grid)
    assert grid.in_flight().size == 0  # a batch traces with an infinite speed of light
    with pytest.raises(native.RtError):
        native.rt_batch_trace(batch.h, native.trace_params(light_cm=1.0, **synth.DEFAULT_PARAMS))
    batch.close()
    grid.close()


def test_queue_growth_keeps_the_packages_in_flight():
    """A trace whose children overflow the first automatic queue (2^20 records)
    is redone with a larger queue; the redo starts from the same packages in
    flight and halting radii, and the sequence still equals the oracle's."""
    N = 48
    g = synth.pulse(N)
    rng = np.random.default_rng(9)
    pos, ndot, e, sg = synth.random_sources((N, N, N), g["box_len_cm"] / N, 24, 1e52, 1e54, rng)
    g.update(pos_cm=pos, ndot=ndot, e_ph_eV=e, sigma_cm2=sg)
    light = 14.0 * g["box_len_cm"] / N
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    fl = oracle.Flight()
    for step in range(2):
        b = grid.trace(checksums=True, light_cm=light, level0=2, phi_c=5.1, f_term=1e-10, max_level=14)
        o = _oracle(g, fl, light, level0=2)
        _compare_step(g, b, grid.rates(), o, "fp32_mixed")
        _compare_flight(g, grid.in_flight(), fl.packages, "fp32_mixed")
        if step == 1:
            assert b["queue_pushed"] > (1 << 20)  # more children than the first queue held
    grid.close()
