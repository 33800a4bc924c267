"""The allocation-free trace entry point (rt_trace_noalloc).

It exists for callers that cannot allocate device memory: applications whose
device memory is owned by a host framework (an arena or a caching allocator
with a fixed budget), and callers that must not let cudaMalloc or cudaFree
synchronise the device or change its memory footprint.  It keeps its scratch
in a fixed-size static device array instead.

Its results must equal those of the regular entry point (rt_trace on a
library-owned grid) within the FP32-mixed tolerance, on two calls in a row
that share that static array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _device_grid(g):
    n_H = torch.tensor(g["n_H"], dtype=torch.float64, device="cuda")
    x_HI = torch.tensor(g["x_HI"], dtype=torch.float64, device="cuda")
    n_HI = torch.tensor((g["n_H"] * g["x_HI"]).astype(np.float32), device="cuda")
    ncell = int(np.prod(g["dims"]))
    kph = torch.empty(ncell, dtype=torch.float32, device="cuda")
    gamma = torch.empty(ncell, dtype=torch.float32, device="cuda")
    return n_HI, n_H, x_HI, kph, gamma


def _small_clumpy():
    rng = np.random.default_rng(42)
    N = 40
    box = synth.box_cm(N)
    dx = box / N
    pos, ndot, e, sg = synth.random_sources((N, N, N), dx, 30, 1e48, 1e50, rng)
    return synth._grid(N, box, synth.lognormal_density(N, mean=3e-3, seed=42), 1.0, pos, ndot, e, sg)


@pytest.mark.parametrize("make", [lambda: synth.stromgren(32), _small_clumpy], ids=["stromgren32", "clumpy40"])
def test_noalloc_matches_regular_entry_point_twice(make):
    g = make()
    grid = native.Grid(parity.ctx(), g, "fp32_mixed")
    ref = grid.trace(checksums=True, **synth.DEFAULT_PARAMS)
    ref_rates = grid.rates()
    grid.close()
    params = native.trace_params(checksums=True, **synth.DEFAULT_PARAMS)
    n_HI, n_H, x_HI, kph, gamma = _device_grid(g)
    mask = ref_rates["kph"] > 1e-8 * ref_rates["kph"].max()
    for call in range(2):
        b = native.rt_trace_noalloc(g["dims"], g["box_len_cm"], n_HI, n_H, x_HI, kph, gamma, g["pos_cm"],
                                    g["ndot"], g["e_ph_eV"], g["sigma_cm2"], params)
        torch.cuda.synchronize()
        assert b["status"] == 0
        np.testing.assert_array_equal(b["counts"], ref["counts"])
        np.testing.assert_array_equal(b["hashes"], ref["hashes"])
        for key in ("emitted", "absorbed", "escaped"):
            assert abs(b[key] - ref[key]) <= 1e-9 * ref["emitted"], (call, key)
        k = kph.double().cpu().numpy()
        gm = gamma.double().cpu().numpy()
        np.testing.assert_allclose(k[mask], ref_rates["kph"][mask], rtol=parity.TOL["fp32_mixed"])
        if np.all(np.asarray(g["e_ph_eV"]) == 13.6):
            # photons at the threshold heat nothing (Eq. "gamma")
            assert not np.any(gm) and not np.any(ref_rates["gamma"])
        else:
            heated = mask & (ref_rates["gamma"] > 0)
            assert heated.sum() > 0.9 * mask.sum()
            np.testing.assert_allclose(gm[heated], ref_rates["gamma"][heated], rtol=parity.TOL["fp32_mixed"],
                                       atol=0)
            assert not np.any(gm[~mask & (ref_rates["gamma"] == 0)])


def test_noalloc_matches_the_oracle():
    """The allocation-free trace against the FP64 oracle on the same medium:
    counts and checksums exact, k_ph and Gamma within the FP32-mixed tolerance
    in every cell receiving more than 1e-8 of the emitted photons."""
    g = _small_clumpy()
    o = parity.run_oracle(g)
    n_HI, n_H, x_HI, kph, gamma = _device_grid(g)
    b = native.rt_trace_noalloc(g["dims"], g["box_len_cm"], n_HI, n_H, x_HI, kph, gamma, g["pos_cm"], g["ndot"],
                                g["e_ph_eV"], g["sigma_cm2"], native.trace_params(checksums=True,
                                                                                 **synth.DEFAULT_PARAMS))
    torch.cuda.synchronize()
    r = {"kph": kph.double().cpu().numpy(), "gamma": gamma.double().cpu().numpy()}
    worst = parity.assert_trace_parity(g, b, r, o, "fp32_mixed")
    assert worst["gamma"] <= parity.TOL["fp32_mixed"]


def test_noalloc_rejects_sizes_beyond_its_limits():
    g = synth.stromgren(16)
    n_HI, n_H, x_HI, kph, gamma = _device_grid(g)
    params = native.trace_params(**synth.DEFAULT_PARAMS)
    n = 1025  # one more than RT_NOALLOC_MAX_SOURCES
    pos = np.zeros((n, 3))
    with pytest.raises(native.RtError) as e:
        native.rt_trace_noalloc(g["dims"], g["box_len_cm"], n_HI, n_H, x_HI, kph, gamma, pos,
                                np.full(n, 1e48), np.full(n, 13.6), np.full(n, 6.3e-18), params)
    assert e.value.code == native.RT_ERR_INVALID_ARG and "1024" in str(e.value)
    # a trace needing more queue records than the static queue holds is refused, not truncated
    g = synth.stromgren_snapshot(128)
    n_HI, n_H, x_HI, kph, gamma = _device_grid(g)
    with pytest.raises(native.RtError) as e:
        native.rt_trace_noalloc(g["dims"], g["box_len_cm"], n_HI, n_H, x_HI, kph, gamma, g["pos_cm"],
                                g["ndot"], g["e_ph_eV"], g["sigma_cm2"], params)
    assert e.value.code == native.RT_ERR_QUEUE_OVERFLOW
