"""Pins for the oracle's ray tracer (Sec. 2.1-2.2; Steps 1-5 of Sec. 3.1).

Each check compares the oracle with something computed another way: slab
intersection of a ray with every cell, enumeration of the split tree from the
sorted plane crossings, the inverse-square law in an optically thin medium,
global photon conservation, and single-ray attenuation walked by the slab
method.
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1012_2865_gb300 import synth


def _rand_dirs(rng, m):
    v = rng.standard_normal((m, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("dims", [(2, 2, 2), (5, 3, 4), (8, 8, 8)])
def test_dda_matches_slab_intersection(dims):
    rng = np.random.default_rng(11 + sum(dims))
    dirs = list(_rand_dirs(rng, 40))
    # axis-aligned, in-plane and diagonal rays
    dirs += [np.array(d, float) for d in [(1, 0, 0), (0, -1, 0), (0, 0, 1), (1, 1, 0), (-1, 1, 1)]]
    dirs = [d / np.linalg.norm(d) for d in dirs]
    for d in dirs:
        s = rng.uniform(0.05, 0.95, 3) * np.asarray(dims)
        r0 = rng.uniform(0, 0.5)
        cells, dr, r = oracle.ray_path(dims, s, d, r0)
        pos = dr > 0
        bc, bin_, bout = brute.slab_segments(dims, s, d, r0)
        np.testing.assert_array_equal(cells[pos], bc)
        np.testing.assert_allclose(dr[pos], bout - bin_, rtol=1e-12, atol=1e-12)
        # segments tile the path: sum of lengths = distance to the box boundary
        np.testing.assert_allclose(dr.sum(), max(0.0, brute.box_exit(dims, s, d) - r0), rtol=1e-12)


def test_dda_corner_source_face_rays():
    """A ray lying in a boundary plane (n_i = 0, s_i = 0) stays inside (tie-break rule)."""
    dims = (4, 4, 4)
    cells, dr, _ = oracle.ray_path(dims, [0.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    np.testing.assert_array_equal(cells, [[i, 0, 0] for i in range(4)])
    np.testing.assert_allclose(dr, 1.0)
    cells, dr, _ = oracle.ray_path(dims, [0.0, 0.0, 0.0], [0.0, -1.0, 0.0])
    assert len(cells) == 0  # leaves immediately


def _run(g, **kw):
    p = dict(synth.DEFAULT_PARAMS)
    p.update(kw)
    return oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"],
                        g["e_ph_eV"], g["sigma_cm2"], **p)


def _transparent(N, src_idx):
    g = synth.stromgren(N)
    g["n_H"] = g["n_H"] * 0.0
    dx = g["box_len_cm"] / N
    g["pos_cm"] = synth.cell_centre_cm(np.array([src_idx]), dx)
    return g


@pytest.mark.parametrize("N,src,phi_c", [(12, (6, 6, 6), 5.1), (10, (2, 7, 4), 3.1), (9, (0, 0, 8), 10.1)])
def test_split_tree_matches_enumeration(N, src, phi_c):
    g = _transparent(N, src)
    r = _run(g, phi_c=phi_c, max_level=8)
    s = np.asarray(src) + 0.5
    created = brute.split_tree((N, N, N), s, lambda l, p: oracle.pix2vec(l, [p])[0], 1, phi_c, 8)
    counts = np.array([len(created.get(l, ())) for l in range(15)], dtype=np.uint64)
    np.testing.assert_array_equal(r["counts"], counts)
    # every package reaches the boundary in a transparent medium
    b = r["budget"]
    assert b[1] == 0.0
    np.testing.assert_allclose(b[2], b[0], rtol=1e-13)


def test_counts_each_pixel_once():
    """The checksum of the created (level, pixel) set equals that of the enumerated set."""
    g = _transparent(10, (3, 5, 6))
    r = _run(g, max_level=9)
    created = brute.split_tree((10, 10, 10), np.array([3.5, 5.5, 6.5]),
                               lambda l, p: oracle.pix2vec(l, [p])[0], 1, 5.1, 9)
    for l in range(10):
        assert int(r["counts"][l]) == len(created[l])


@pytest.mark.parametrize("seed", [0, 1])
def test_photon_conservation_and_deposit_identity(seed):
    """emitted = absorbed + escaped (1e-12), and sum_c k_c n_HI,c V = absorbed."""
    rng = np.random.default_rng(seed)
    N = 20
    g = synth.clumpy(N=N, nsrc=5, seed=100 + seed)
    g["x_HI"] = rng.uniform(0.0, 1.0, N ** 3)
    g["x_HI"][rng.random(N ** 3) < 0.1] = 0.0  # fully ionised cells
    r = _run(g)
    b = r["budget"]
    np.testing.assert_allclose(b[0], g["ndot"].sum(), rtol=1e-14)
    assert abs(b[0] - b[1] - b[2]) <= 1e-12 * b[0]
    dx = g["box_len_cm"] / N
    nHI = g["n_H"] * g["x_HI"]
    dep = np.sum(r["kph"] * nHI) * dx ** 3
    np.testing.assert_allclose(dep, b[1], rtol=1e-12)
    # Gamma = k_ph (E - 13.6 eV) per source: check with one source at a time
    for s in range(2):
        g1 = dict(g)
        for key in ("pos_cm", "ndot", "e_ph_eV", "sigma_cm2"):
            g1[key] = g[key][s:s + 1]
        r1 = _run(g1)
        np.testing.assert_allclose(r1["gamma"], r1["kph"] * (g1["e_ph_eV"][0] - 13.6) * 1.602176634e-12,
                                   rtol=1e-13)


def test_opaque_medium_absorbs_everything():
    g = synth.stromgren(16)
    g["n_H"] = synth.round_f32(np.full(16 ** 3, 1.0))  # tau per cell ~ 6e2
    g["pos_cm"] = synth.cell_centre_cm(np.array([[8, 8, 8]]), g["box_len_cm"] / 16)
    r = _run(g)
    b = r["budget"]
    assert b[2] == 0.0
    assert abs(b[0] - b[1]) <= 1e-12 * b[0]
    # only the source cell and its neighbours receive radiation
    assert np.count_nonzero(r["kph"]) <= 27


def test_single_rays_against_slab_walk():
    """No splitting (tiny Phi_c): each of the 12 level-0 rays attenuates along its slab path."""
    dims = (7, 5, 6)
    g = synth.stromgren(7)
    g["dims"] = dims
    ncell = 7 * 5 * 6
    rng = np.random.default_rng(3)
    g["n_H"] = synth.round_f32(rng.uniform(0.0, 2e-3, ncell))
    g["x_HI"] = rng.uniform(0.2, 1.0, ncell)
    dx = g["box_len_cm"] / 7
    src = np.array([2.3, 1.7, 3.9])
    g["pos_cm"] = (src * dx).reshape(1, 3)
    s_cells = g["pos_cm"][0] / dx
    r = _run(g, level0=0, phi_c=1e-8)
    assert r["counts"][0] == 12 and r["counts"][1:].sum() == 0
    # base directions from the closed-form layout: z in {2/3, 0, -2/3}
    zs = [2 / 3] * 4 + [0.0] * 4 + [-2 / 3] * 4
    phis = [(2 * k + 1) * np.pi / 4 for k in range(4)] + [k * np.pi / 2 for k in range(4)] + \
           [(2 * k + 1) * np.pi / 4 for k in range(4)]
    k_ref = np.zeros(ncell)
    P0 = g["ndot"][0] / 12
    sigma = g["sigma_cm2"][0]
    nHI = g["n_H"] * g["x_HI"]
    for z, ph in zip(zs, phis):
        st = np.sqrt(1 - z * z)
        n = np.array([st * np.cos(ph), st * np.sin(ph), z])
        n[np.abs(n) < 1e-15] = 0.0
        cells, tin, tout = brute.slab_segments(dims, s_cells, n)
        P = P0
        tau_tot = 0.0
        for (ci, cj, ck), a, b in zip(cells, tin, tout):
            idx = ci + dims[0] * (cj + dims[1] * ck)
            tau = sigma * nHI[idx] * (b - a) * dx
            dP = P * (1 - np.exp(-tau))
            k_ref[idx] += P * sigma * (b - a) * dx / dx ** 3 * (1.0 if tau == 0 else (1 - np.exp(-tau)) / tau)
            P -= dP
            tau_tot += tau
            if P < 1e-10 * P0:  # package spent: the rest is absorbed where it stands
                k_ref[idx] += P / (nHI[idx] * dx ** 3)
                break
    np.testing.assert_allclose(r["kph"], k_ref, rtol=1e-9, atol=1e-12 * k_ref.max())


def _thin_scatter(N, phi_c, src):
    g = synth.stromgren(N)
    g["n_H"] = synth.round_f32(np.full(N ** 3, 1e-3))
    g["x_HI"] = np.full(N ** 3, 1e-8)
    dx = g["box_len_cm"] / N
    g["pos_cm"] = synth.cell_centre_cm(np.array([src]), dx)
    r = _run(g, phi_c=phi_c)
    i = np.arange(N) + 0.5
    X = (i[None, None, :] - (src[0] + 0.5)) ** 2 + (i[None, :, None] - (src[1] + 0.5)) ** 2 + \
        (i[:, None, None] - (src[2] + 0.5)) ** 2
    rc = np.sqrt(X).reshape(-1) * dx
    sel = (rc > 3 * dx) & (rc < (N / 2 - 2) * dx)
    k_thin = g["sigma_cm2"][0] * g["ndot"][0] / (4 * np.pi * rc[sel] ** 2)
    return r["kph"][sel] / k_thin - 1.0


def test_optically_thin_inverse_square():
    """In a transparent medium k_ph follows sigma Ndot / (4 pi r^2) (Sec. 7.2).

    The scatter about the inverse-square law falls as Phi_c grows; the paper
    finds sigma ~ Phi_c^-0.6 independent of resolution.
    """
    stds = []
    phis = [1.1, 2.1, 5.1, 10.1, 25.1]
    for pc in phis:
        dev = _thin_scatter(32, pc, (15, 16, 14))
        assert abs(np.mean(dev)) < 0.05, (pc, np.mean(dev))
        stds.append(np.std(dev))
    slope = np.polyfit(np.log(phis), np.log(stds), 1)[0]
    # the paper's -0.6 is with its covering-factor correction on; without it
    # the slope is measured near -0.7: the bound proposed for this pin
    assert -0.9 < slope < -0.3, (slope, stds)
    assert stds[-1] < stds[0]


def test_stromgren_constants_golden():
    """Test 1 parameters give the paper's R_s = 5.4 kpc and t_rec = 122.4 Myr."""
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "test1_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                vals[k] = float(v)
    Rs = (3 * vals["ndot"] / (4 * np.pi * vals["alpha_B"] * vals["n_H"] ** 2)) ** (1 / 3)
    trec = 1.0 / (vals["alpha_B"] * vals["n_H"])
    assert abs(Rs / synth.KPC_CM - vals["R_s_kpc"]) < 0.05
    assert abs(trec / synth.MYR_S - vals["t_rec_Myr"]) < 0.1


def test_root_ranges_sum_to_the_whole_trace():
    """The trace is a sum over root packages: disjoint root ranges that cover
    every root give, summed, the counts, checksums and segments of the whole
    pass exactly and its k_ph, Gamma and budget up to summation order."""
    g = synth.clumpy(16, 5)
    args = (g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"], g["sigma_cm2"])
    whole = oracle.trace(*args, **synth.DEFAULT_PARAMS)
    nroots = 5 * 48
    cuts = [0, 1, 47, 48, 130, 239, nroots]
    parts = [oracle.trace_roots(*args, a, b - a, **synth.DEFAULT_PARAMS) for a, b in zip(cuts[:-1], cuts[1:])]
    assert np.array_equal(sum(p["counts"] for p in parts), whole["counts"])
    assert np.array_equal(sum(p["hashes"] for p in parts), whole["hashes"])
    assert sum(p["segments"] for p in parts) == whole["segments"]
    for key in ("kph", "gamma"):
        tot = sum(p[key] for p in parts)
        m = whole[key] > 0
        assert np.array_equal(tot > 0, m)
        assert np.max(np.abs(tot[m] - whole[key][m]) / whole[key][m]) < 1e-12
    assert np.allclose(sum(p["budget"] for p in parts), whole["budget"], rtol=1e-12, atol=0)
    # an empty range does nothing; a range past the last root is cut at it
    empty = oracle.trace_roots(*args, nroots, 10, **synth.DEFAULT_PARAMS)
    assert empty["segments"] == 0 and not np.any(empty["kph"]) and empty["budget"][0] == 0
