"""The finite-speed-of-light benchmark configuration at full size (Application 5:
128^3 cells, 1 Mpc, pulsed corner source, dt_P = 50 kyr), FP32-mixed, in the
launch configuration the benchmark times.

* the first steps against the oracle's steps (each side with its own packages
  in flight and its own chemistry): counts, checksums, budget, k_ph, and the
  packages in flight;
* every step of the 6 Myr run: photons conserved with the packages resumed
  and halted, and what one step halts the next resumes;
* after 6 Myr (light has crossed the box): in every radial band of width
  c dt_P within the optically thin inner 80 cells, the flux follows the
  inverse-square law with the source's rate at that band's emission time
  (Eq. "test12"), the property the paper's figure of Application 5 shows.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


def test_application5_pulse_full_size():
    g = synth.pulse(128)
    N = 128
    dt, light = g["dt_s"], g["light_cm"]
    dx = g["box_len_cm"] / N
    c_dt = light / dx
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    fl = oracle.Flight()
    x, z = g["x_HI"].copy(), g["x_HII"].copy()
    prev = None
    n_steps = int(round(6.0 * synth.MYR_S / dt))
    for n in range(n_steps):
        rate = np.array([float(synth.pulse_rate(n * dt))])
        grid.set_source_rates(rate)
        b = grid.trace(checksums=True, light_cm=light, **synth.DEFAULT_PARAMS)
        assert b["status"] == 0
        lhs = b["emitted"] + b["resumed"]
        assert abs(lhs - b["absorbed"] - b["escaped"] - b["halted"]) <= 1e-12 * lhs
        if prev is not None:
            assert b["n_resumed"] == prev["n_halted"]
            assert abs(b["resumed"] - prev["halted"]) <= 1e-12 * prev["halted"]
        prev = b
        if n < 4:  # the oracle follows the first steps
            go = dict(g, x_HI=x, ndot=rate)
            o = oracle.trace(go["dims"], go["box_len_cm"], go["n_H"], go["x_HI"], go["pos_cm"], go["ndot"],
                             go["e_ph_eV"], go["sigma_cm2"], flight=fl, light_cm=light, **synth.DEFAULT_PARAMS)
            np.testing.assert_array_equal(b["counts"], o["counts"])
            np.testing.assert_array_equal(b["hashes"], o["hashes"])
            assert b["n_halted"] == o["n_halted"]
            total = o["budget"][0] + o["resumed"]
            for got, ref in ((b["absorbed"], o["budget"][1]), (b["escaped"], o["budget"][2]),
                             (b["halted"], o["halted"])):
                assert abs(got - ref) <= parity.BUDGET_TOL["fp32_mixed"] * total
            k = grid.rates()["kph"]
            m = parity.receiving_mask(go, o["kph"], total)
            rel = np.abs(k[m] - o["kph"][m]) / o["kph"][m]
            assert rel.max() <= parity.TOL["fp32_mixed"]
            got = grid.in_flight()
            assert got.size == fl.packages.size
            np.testing.assert_allclose(np.sort(got["r_cm"] / dx), np.sort(fl.packages["r"]), rtol=1e-12)
            x, z = oracle.chem(g["n_H"], x, z, o["kph"], dt, 10, synth.ALPHA_B)
        grid.chem(dt, 10, synth.ALPHA_B)
    assert prev["n_halted"] > 10_000_000  # packages of every age fill the box
    # Application 5: the flux in each band follows 1/r^2 with that band's emission rate
    i = np.arange(N, dtype=np.float64) + 0.5
    R = np.sqrt(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2).reshape(-1)
    age = np.floor(R / c_dt).astype(int)
    inner = np.abs(R - (age + 0.5) * c_dt) < 0.5 * c_dt - 0.9  # cells wholly inside a band
    k = grid.rates()["kph"]
    q = k * (R * dx) ** 2 * 4.0 * np.pi / g["sigma_cm2"][0]  # the rate the cell sees, photons/s
    ratio = []
    for a in range(3, age.max() + 1):
        # within 80 cells the gas stays optically thin over the 6 Myr (farther out the
        # dark phases let it recombine to tau ~ 0.3, which the update couples back)
        m = inner & (age == a) & (R < 80.0)
        if m.sum() < 50:
            continue
        emitted = float(synth.pulse_rate((n_steps - 1 - a) * dt))
        ratio.append(np.median(q[m]) / emitted)
    ratio = np.array(ratio)
    assert ratio.size > 20
    np.testing.assert_allclose(ratio, 1.0, atol=0.1)
    grid.close()
