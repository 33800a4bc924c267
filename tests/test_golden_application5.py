"""The Application 5 workload against the parameters the paper prints
(tests/golden/application5.txt, Sec. 9 and Eq. "test12"), and the pulse
shape of Eq. "test12": period t0, peak L_max at t0/2 + k t0, minimum
L_max e^-A at multiples of t0."""
import os

import numpy as np

from paper_1012_2865_gb300 import synth

KPC = synth.KPC_CM


def _golden():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "application5.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if len(line) == 2:
                vals[line[0]] = float(line[1])
    return vals


def test_workload_uses_the_printed_parameters():
    v = _golden()
    g = synth.pulse(128)
    assert abs(g["box_len_cm"] / (1000.0 * KPC) - v["L_box_Mpc"]) < 1e-5
    assert np.all(g["n_H"] == np.float32(v["rho_cm3"]))
    assert g["dt_s"] == v["dt_P_kyr"] * 1e-3 * synth.MYR_S
    # the printed light-crossing time of the box
    crossing = g["box_len_cm"] / synth.C_CM_S / synth.MYR_S
    assert abs(crossing - v["crossing_Myr"]) < 0.05
    # light crosses 1/65 of the box per step, 120 steps in the printed run
    assert abs(g["light_cm"] / g["box_len_cm"] - v["dt_P_kyr"] * 1e-3 / crossing) < 1e-3
    assert round(v["run_Myr"] / (v["dt_P_kyr"] * 1e-3)) == 120


def test_pulse_shape_of_eq_test12():
    v = _golden()
    t0 = v["t0_Myr"] * synth.MYR_S
    L = lambda t: float(synth.pulse_rate(t, L_max=v["L_max_ph_s"], t0_s=t0, A=v["A"]))  # noqa: E731
    for k in range(4):
        assert abs(L((k + 0.5) * t0) / v["L_max_ph_s"] - 1.0) < 1e-12  # peaks
        assert abs(L(k * t0) / (v["L_max_ph_s"] * np.exp(-v["A"])) - 1.0) < 1e-12  # troughs
    t = np.linspace(0.0, 3.0 * t0, 301)
    np.testing.assert_allclose(synth.pulse_rate(t + t0, t0_s=t0), synth.pulse_rate(t, t0_s=t0), rtol=1e-9)
    # symmetric about each peak
    np.testing.assert_allclose(synth.pulse_rate(0.5 * t0 + t[:50], t0_s=t0),
                               synth.pulse_rate(0.5 * t0 - t[:50], t0_s=t0), rtol=1e-9)
