"""Pins for the finite speed of light in the oracle (Sec. 2.1, halting
condition 1; Step 3j; Application 5, Eq. "test12").

A package travels c dt_P per trace and is then kept, with its cell, for the
next trace, which continues it through the medium of that step.  What fixes
the result independently of the halting code:

* light that outruns the box changes nothing (bit-identical trace);
* after the first trace, a cell wholly nearer the source than c dt_P holds
  exactly the infinite-speed rates, and no cell wholly beyond it is reached;
* in a static medium with a constant source the traces reach a steady state
  equal to the infinite-speed trace: once every age up to the box diagonal is
  in flight, the packages alive in one trace are the infinite trace cut into
  radial bands, so rates, packages per level and the created-set checksum
  are those of one infinite trace (a split segment deposits
  P (1 - e^-t1) + P e^-t1 (1 - e^-t2) = P (1 - e^-(t1 + t2)));
* one emission followed by dark traces delivers exactly the photons, and the
  rates summed over the traces, of the infinite trace;
* the rates are linear in each emission's rate, so a rate change between
  traces reweights only the new packages;
* Application 5: in an optically thin box the flux in each band of width
  c dt_P follows the inverse-square law with the rate at that band's
  emission time (Eq. "test12"): shells of the pulse travel outwards;
* emitted + resumed = absorbed + escaped + halted in every trace.
"""
import numpy as np

import oracle
from paper_1012_2865_gb300 import synth


def _trace(g, **kw):
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], **kw)


def _conserves(r):
    b = r["budget"]
    lhs = b[0] + r["resumed"]
    rhs = b[1] + b[2] + r["halted"]
    assert abs(lhs - rhs) <= 1e-12 * max(lhs, 1e-300), (lhs, rhs)


def _static(N=16, nsrc=3, seed=4):
    g = synth.clumpy(N=N, nsrc=nsrc, seed=seed)
    g["x_HI"] = np.full(N ** 3, 0.02)  # optical depth ~0.3-1 per cell: terminations and long rays
    return g


def _diag(g):
    return float(np.sqrt(np.sum(np.asarray(g["dims"], dtype=np.float64) ** 2)))


def test_light_beyond_the_box_changes_nothing():
    g = _static()
    dx = g["box_len_cm"] / g["dims"][0]
    inf = _trace(g)
    fl = oracle.Flight()
    fin = _trace(g, flight=fl, light_cm=2.0 * _diag(g) * dx)
    for key in ("kph", "gamma", "budget", "counts", "hashes"):
        np.testing.assert_array_equal(fin[key], inf[key], err_msg=key)
    assert fin["segments"] == inf["segments"]
    assert fin["n_halted"] == 0 and fin["halted"] == 0.0 and fin["resumed"] == 0.0


def test_first_trace_reaches_only_the_light_front():
    N = 24
    g = synth.pulse(N)
    g["ndot"] = np.array([1e55])
    dx = g["box_len_cm"] / N
    c_dt = 9.3
    inf = _trace(g)
    fl = oracle.Flight()
    fin = _trace(g, flight=fl, light_cm=c_dt * dx)
    _conserves(fin)
    i = np.arange(N, dtype=np.float64)
    lo = np.sqrt(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2).reshape(-1)  # nearest corner
    hi = np.sqrt(((i + 1)[:, None, None]) ** 2 + ((i + 1)[None, :, None]) ** 2 + ((i + 1)[None, None, :]) ** 2).reshape(-1)
    inside, beyond = hi < c_dt, lo > c_dt
    assert inside.sum() > 100 and beyond.sum() > 1000
    np.testing.assert_array_equal(fin["kph"][inside], inf["kph"][inside])
    assert np.all(fin["kph"][beyond] == 0.0)
    assert np.all(inf["kph"][beyond] > 0.0)
    # every halted package sits on the light front, in its cell
    f = fl.packages
    assert f.size == fin["n_halted"] > 0
    assert np.all(f["r"] == c_dt) and np.all(f["age"] == 1)
    for k in range(0, f.size, max(1, f.size // 200)):
        p = c_dt * oracle.pix2vec(int(f["level"][k]), [int(f["pix"][k])])[0]  # source at the origin
        np.testing.assert_array_equal(f["cell"][k], np.floor(p))


def test_steady_state_equals_the_infinite_trace():
    g = _static()
    dx = g["box_len_cm"] / g["dims"][0]
    c_dt = 3.3
    inf = _trace(g)
    fl = oracle.Flight()
    M = int(np.ceil(_diag(g) / c_dt)) + 2
    for _ in range(M):
        r = _trace(g, flight=fl, light_cm=c_dt * dx)
        _conserves(r)
    np.testing.assert_array_equal(r["counts"], inf["counts"])
    np.testing.assert_array_equal(r["hashes"], inf["hashes"])
    assert r["segments"] > inf["segments"]  # segments cut at the band edges
    for key in ("kph", "gamma"):
        ref = inf[key]
        m = ref > 1e-14 * ref.max()
        np.testing.assert_allclose(r[key][m], ref[m], rtol=1e-10)
        assert np.all(r[key][~m] <= 1e-12 * ref.max())
    em = inf["budget"][0]
    assert abs(r["budget"][1] - inf["budget"][1]) <= 1e-12 * em
    assert abs(r["budget"][2] - inf["budget"][2]) <= 1e-12 * em
    assert abs(r["resumed"] - r["halted"]) <= 1e-12 * em  # as many photons leave flight as enter it
    assert r["n_halted"] == fl.packages.size > 0
    # halting radii: the light travel since emission, summed in order
    assert np.all(np.diff(fl.rlim) > 0) and abs(fl.rlim[M - 1] - M * c_dt) <= 1e-12 * M * c_dt


def test_one_emission_is_delivered_once():
    g = _static(seed=8)
    dx = g["box_len_cm"] / g["dims"][0]
    c_dt = 2.7
    inf = _trace(g)
    fl = oracle.Flight()
    ndot = g["ndot"].copy()
    k_sum = np.zeros_like(inf["kph"])
    g_sum = np.zeros_like(inf["gamma"])
    out = 0.0
    M = int(np.ceil(_diag(g) / c_dt)) + 2
    for m in range(M):
        g["ndot"] = ndot if m == 0 else np.zeros_like(ndot)  # dark after the first step
        r = _trace(g, flight=fl, light_cm=c_dt * dx)
        _conserves(r)
        k_sum += r["kph"]
        g_sum += r["gamma"]
        out += r["budget"][1] + r["budget"][2]
    assert r["halted"] == 0.0
    em = inf["budget"][0]
    assert abs(out - em) <= 1e-12 * em
    for got, ref in ((k_sum, inf["kph"]), (g_sum, inf["gamma"])):
        m = ref > 1e-14 * ref.max()
        np.testing.assert_allclose(got[m], ref[m], rtol=1e-10)


def test_rate_change_reweights_only_new_packages():
    g = _static(seed=12)
    dx = g["box_len_cm"] / g["dims"][0]
    c_dt = 4.1
    n1 = g["ndot"].copy()
    n2 = n1 * np.array([0.25, 3.0, 1.0])[: n1.size]
    const = oracle.Flight()
    _trace(g, flight=const, light_cm=c_dt * dx)
    k2c = _trace(g, flight=const, light_cm=c_dt * dx)["kph"]
    fl = oracle.Flight()
    _trace(g, flight=fl, light_cm=c_dt * dx)
    g["ndot"] = n2
    r2 = _trace(g, flight=fl, light_cm=c_dt * dx)
    _conserves(r2)
    # K2 = K(new packages at n2) + K(resumed at n1), and each source's first-trace
    # field is linear in its rate
    single = []
    for s in range(n1.size):
        gs = dict(g)
        gs["ndot"] = np.where(np.arange(n1.size) == s, n1, 0.0)
        single.append(_trace(gs, flight=oracle.Flight(), light_cm=c_dt * dx)["kph"])
    expect = k2c + sum((n2[s] / n1[s] - 1.0) * single[s] for s in range(n1.size))
    np.testing.assert_allclose(r2["kph"], expect, rtol=0, atol=1e-11 * k2c.max())
    assert not np.allclose(r2["kph"], k2c, rtol=1e-3, atol=0.0)


def test_pulse_shells_follow_the_source_history():
    """Application 5: inverse-square flux in each band with that band's emission rate."""
    N = 32
    g = synth.pulse(N)
    dx = g["box_len_cm"] / N
    c_dt = 4.0
    dt = 0.2 * synth.MYR_S   # light_cm fixed by c_dt below; t0 = 10 steps as in the paper
    t0 = 10 * dt
    fl = oracle.Flight()
    n_steps = int(np.ceil(_diag(g) / c_dt)) + 1
    for n in range(n_steps):
        g["ndot"] = np.array([float(synth.pulse_rate(n * dt, t0_s=t0))])
        r = _trace(g, flight=fl, light_cm=c_dt * dx)
        _conserves(r)
    i = np.arange(N, dtype=np.float64) + 0.5
    R = np.sqrt(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2).reshape(-1)
    age = np.floor(R / c_dt).astype(int)
    interior = np.abs(R - (age + 0.5) * c_dt) < 0.5 * c_dt - 0.9  # cell wholly inside its band
    q = r["kph"] * (R * dx) ** 2 * 4.0 * np.pi / g["sigma_cm2"][0]  # = rate seen, photons/s
    seen, emitted = [], []
    for a in range(1, age.max() + 1):
        m = interior & (age == a) & (R > 5.0)
        if m.sum() < 20:
            continue
        seen.append(np.median(q[m]))
        emitted.append(float(synth.pulse_rate((n_steps - 1 - a) * dt, t0_s=t0)))
    seen, emitted = np.array(seen), np.array(emitted)
    assert emitted.max() / emitted.min() > 20  # the bands span most of the pulse
    np.testing.assert_allclose(seen / emitted, 1.0, atol=0.1)
