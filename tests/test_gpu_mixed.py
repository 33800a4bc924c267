"""FP32-mixed CUDA path vs the FP64 oracle (through the C ABI).

Counts per level and the created-set checksum must be bit-exact (the mixed
walker re-takes every uncertain decision in FP64); k_ph and Gamma within 1e-3
relative in cells receiving > 1e-8 of the emitted photons; the FP64 photon
budget conserves photons to 1e-12.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1012_2865_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level", [0, 1, 2, 4, 6, 8, 10])
def test_fp32_direction_bound_holds(level):
    err, bound = native.rt_selfcheck_directions(parity.ctx(), level)
    assert err <= 0.5 * bound, (level, err, bound)


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_update_matches_oracle_on_the_same_rates(precision):
    """The ionisation update alone: given the rates this grid's own trace
    deposited, the GPU update equals the oracle's to rounding (FP64: the same
    operations; FP32-mixed: double-float Newton corrections, ~1e-13)."""
    g = synth.clumpy(N=32, nsrc=20, seed=5)
    rng = np.random.default_rng(3)
    g["x_HI"] = np.where(rng.random(32 ** 3) < 0.5, 1.0, 10.0 ** rng.uniform(-9, 0, 32 ** 3))
    g["x_HII"] = 1.0 - g["x_HI"]
    grid, b, r = parity.run_gpu(g, precision)
    grid.chem(synth.MYR_S, 10, synth.ALPHA_B)
    x_gpu = grid.rates()["x_HI"]
    x_o, z_o = oracle.chem(g["n_H"], g["x_HI"], g["x_HII"], np.asarray(r["kph"], dtype=np.float64), synth.MYR_S, 10,
                           synth.ALPHA_B)
    rtol = 1e-14 if precision == "fp64" else 1e-11
    np.testing.assert_allclose(x_gpu, x_o, rtol=rtol, atol=1e-300)
    np.testing.assert_allclose(1.0 - x_gpu[x_gpu < 0.5], z_o[x_gpu < 0.5], rtol=1e-9)
    grid.close()


def test_config0_mixed():
    g = synth.stromgren(32)
    grid, b, r = parity.run_gpu(g, "fp32_mixed")
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o, "fp32_mixed")
    grid.chem(synth.MYR_S, 10, synth.ALPHA_B)
    x_o, _ = oracle.chem(g["n_H"], g["x_HI"], g["x_HII"], o["kph"], synth.MYR_S, 10, synth.ALPHA_B)
    np.testing.assert_allclose(grid.rates()["x_HI"], x_o, rtol=1e-3, atol=1e-12)
    grid.close()


@pytest.mark.parametrize("seed,dims,nsrc,level0,phi_c", [
    (0, (24, 24, 24), 6, 1, 5.1),
    (1, (37, 23, 29), 9, 0, 3.1),
    (2, (16, 40, 8), 4, 2, 10.1),
    (3, (48, 48, 48), 20, 1, 5.1),
])
def test_clumpy_ragged_grids_mixed(seed, dims, nsrc, level0, phi_c):
    rng = np.random.default_rng(seed)
    box = 6.6 * synth.KPC_CM * dims[0] / 32
    dx = box / dims[0]
    n = synth.lognormal_density(None, mean=2e-3, seed=seed, dims=dims)
    pos, ndot, e, sg = synth.random_sources(dims, dx, nsrc, 1e48, 1e50, rng)
    g = synth._grid(dims, box, n, rng.uniform(0.0, 1.0, int(np.prod(dims))), pos, ndot, e, sg)
    _, b, r = parity.run_gpu(g, "fp32_mixed", level0=level0, phi_c=phi_c)
    o = parity.run_oracle(g, level0=level0, phi_c=phi_c)
    parity.assert_trace_parity(g, b, r, o, "fp32_mixed")


def test_off_grid_sources_mixed():
    """Source positions that are not exact in FP32 (no structural-tie shortcut)."""
    rng = np.random.default_rng(9)
    dims = (20, 20, 20)
    box = 6.6 * synth.KPC_CM * 20 / 32
    pos = rng.uniform(0.05, 0.95, (5, 3)) * box
    g = synth._grid(dims, box, synth.lognormal_density(None, mean=2e-3, seed=9, dims=dims),
                    rng.uniform(0.0, 1.0, 8000), pos, np.full(5, 1e49), np.full(5, 20.0),
                    np.full(5, synth.SIGMA_HI))
    _, b, r = parity.run_gpu(g, "fp32_mixed")
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o, "fp32_mixed")


def test_partially_ionised_128_mixed():
    g = synth.stromgren_snapshot(128)
    _, b, r = parity.run_gpu(g, "fp32_mixed")
    o = parity.run_oracle(g)
    parity.assert_trace_parity(g, b, r, o, "fp32_mixed")
    # the FP64 path agrees with the oracle bit for bit on the same input
    _, b64, r64 = parity.run_gpu(g, "fp64")
    parity.assert_trace_parity(g, b64, r64, o, "fp64")


def test_stromgren_500myr_mixed_vs_fp64():
    """Coupled 128^3 evolution in both precisions: R_IF within 2 % of R_s and of each other."""
    N = 128
    g = synth.stromgren(N)
    V = (g["box_len_cm"] / N) ** 3
    rs = (3 * 5e48 / (4 * np.pi * synth.ALPHA_B * 1e-3 ** 2)) ** (1 / 3)
    out = {}
    for prec in ("fp32_mixed", "fp64"):
        grid = native.Grid(parity.ctx(), g, prec)
        for s in range(1000):
            grid.trace(sync=False, queue_capacity=1 << 22)
            grid.chem(0.5 * synth.MYR_S, 10, synth.ALPHA_B)
        b = native.rt_get_budget(grid.h)
        assert abs(b["emitted"] - b["absorbed"] - b["escaped"]) <= 1e-12 * b["emitted"]
        z = grid.x_HII()
        r = grid.rates()
        out[prec] = ((6 * np.sum(z) * V / np.pi) ** (1 / 3), r["kph"], r["x_HI"], b)
        grid.close()
    R32, R64 = out["fp32_mixed"][0], out["fp64"][0]
    assert abs(R32 / rs - 1) < 0.02 and abs(R64 / rs - 1) < 0.02, (R32 / rs, R64 / rs)
    assert abs(R32 / R64 - 1) < 1e-3, R32 / R64
    np.testing.assert_array_equal(out["fp32_mixed"][3]["counts"], out["fp64"][3]["counts"])
