"""Seeded synthetic workloads.

This module only draws inputs (media, sources, request streams); it holds none
of the radiative-transfer arithmetic, so the CUDA path and the oracle can both
consume what it produces.  Every array of densities is rounded to values that
FP32 represents exactly, so an FP32 grid and an FP64 grid hold the same medium.

Recipes (base seed 20101, numpy PCG64):

* ``strömgren(N)`` -- Test 1 of Sec. 4.1: box 6.6 kpc, n_H = 1e-3 cm^-3,
  x_HI = 1, T = 1e4 K, one 13.6 eV source of 5e48 photons/s at the corner
  (0, 0, 0), sigma_HI = 6.3e-18 cm^2, alpha_B = 2.59e-13 cm^3/s.
* ``lognormal_density(N)`` -- Gaussian random field g with P(k) ~ k^-3
  (k = 0 removed), unit variance, n = nbar exp(s g) / mean(exp(s g)) with
  s = 1.0 and nbar = 1e-2 cm^-3.  Stands in for the cosmological density
  fields of Test 4 and the reionisation run of Sec. 9, which are not
  available here.
* ``clumpy(N, nsrc)`` -- that medium with ``nsrc`` sources at uniform-random
  cell centres, Ndot log-uniform in [1e48, 1e50] photons/s, photon energies
  uniform in [13.6, 29.6] eV (29.6 eV is the mean energy of the 1e5 K black
  body used in Sec. 7.3), sigma = 6.3e-18 cm^2 for every source.
* ``batch(n_inst)`` -- grid sides drawn from {32, 48, 64, 96, 128, 192}, the
  same medium, 1-256 sources, Ndot log-uniform in [1e47, 1e50].
* ``request_stream(rate, duration)`` -- Poisson arrivals; cells log-uniform in
  [64^3, 256^3], 1-500 sources, 1-20 coupled steps of 0.5 Myr.
* ``typed_clumpy(N=128, nsrc=30)`` -- the clumpy medium with photon types
  (Sec. 3.2): sources cycle through H I, He I and He II ionising, photon energies uniform
  in [E_i, E_i + 16] eV, threshold cross sections 6.3e-18, 7.43e-18 and
  1.58e-18 cm^2; helium at n_He = 0.079 n_H (primordial), 90 % He I and 10 %
  He II.
* ``pulse(N)`` -- Application 5 (Sec. 9): a 1 Mpc box of uniform n_H = 1e-4
  cm^-3, kept optically thin (x_HI = 1e-5, what photo-ionisation equilibrium
  gives there), one 29.6 eV source at the corner whose rate follows
  ``pulse_rate(t)`` (Eq. "test12": L_max = 1e55 photons/s, t0 = 0.5 Myr,
  A = 4); radiative-transfer timestep 50 kyr, so light crosses 1/65 of the
  box per step.
"""
from __future__ import annotations

import numpy as np

KPC_CM = 3.0856775814913673e21
MYR_S = 3.15576e13  # one million Julian years
SIGMA_HI = 6.3e-18
ALPHA_B = 2.59e-13
E_HI_EV = 13.6
BASE_SEED = 20101
C_CM_S = 2.99792458e10  # speed of light

DEFAULT_PARAMS = dict(level0=1, phi_c=5.1, f_term=1e-10, max_level=14)


def box_cm(N: int, box_kpc: float = 6.6) -> float:
    """Box length near box_kpc whose cell width box/N has at most 20 significant
    bits, so every cell centre (i + 1/2) dx is an exact double and divides back
    to exactly i + 1/2 (the relative change of the box is below 1e-6)."""
    dx = box_kpc * KPC_CM / N
    e = np.floor(np.log2(dx)) - 19
    dx = np.round(dx / 2.0 ** e) * 2.0 ** e
    return float(dx * N)


def round_f32(a) -> np.ndarray:
    """float64 array whose values are exactly representable in FP32."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def cell_centre_cm(idx, dx: float) -> np.ndarray:
    """Positions (cm) of cell centres; where a float exists whose quotient by dx is
    exactly i + 1/2 it is chosen, so the centre is exact in cell units."""
    want = np.asarray(idx, dtype=np.float64) + 0.5
    base = want * dx
    out = base.copy()
    flat_w, flat_o = want.reshape(-1), out.reshape(-1)
    for j in range(flat_w.size):
        if flat_o[j] / dx == flat_w[j]:
            continue
        cand = flat_o[j]
        for step in (1, -1, 2, -2, 3, -3, 4, -4):
            c = flat_o[j]
            for _ in range(abs(step)):
                c = np.nextafter(c, np.inf if step > 0 else -np.inf)
            if c / dx == flat_w[j]:
                cand = c
                break
        flat_o[j] = cand
    return out


def _grid(N, box_len_cm, n_H, x_HI, pos_cm, ndot, e_ph, sigma, **extra):
    dims = (N, N, N) if np.isscalar(N) else tuple(int(v) for v in N)
    ncell = dims[0] * dims[1] * dims[2]
    n_H = round_f32(np.broadcast_to(n_H, (ncell,)))
    x_HI = np.array(np.broadcast_to(x_HI, (ncell,)), dtype=np.float64)
    g = dict(dims=dims, box_len_cm=float(box_len_cm), n_H=n_H, x_HI=x_HI,
             x_HII=1.0 - x_HI, pos_cm=np.asarray(pos_cm, dtype=np.float64).reshape(-1, 3),
             ndot=np.asarray(ndot, dtype=np.float64).reshape(-1),
             e_ph_eV=np.asarray(e_ph, dtype=np.float64).reshape(-1),
             sigma_cm2=np.asarray(sigma, dtype=np.float64).reshape(-1))
    g.update(extra)
    return g


def stromgren(N: int = 128, box_kpc: float = 6.6, n_H: float = 1e-3, ndot: float = 5e48) -> dict:
    """Test 1 (Sec. 4.1) on an N^3 grid; source at the domain corner."""
    return _grid(N, box_cm(N, box_kpc), n_H, 1.0, [[0.0, 0.0, 0.0]], [ndot], [13.6], [SIGMA_HI],
                 alpha_B=ALPHA_B)


def stromgren_snapshot(N: int = 128, t_myr: float = 500.0, width_cells: float = 3.0,
                       x_in: float = 1e-3) -> dict:
    """Test 1 medium with an ionised octant sphere at the analytic I-front radius.

    x_HI(r) = x_in + (1 - x_in) / (1 + exp(-(r - r_IF) / w)), r the distance of a
    cell centre from the corner source, r_IF = R_s [1 - exp(-t/t_rec)]^(1/3)
    (Eqs. "Rstr", "rstr"), w = width_cells * N / 128 cells.  A seeded-free,
    deterministic stand-in for the coupled evolution's state at time t.
    """
    g = stromgren(N)
    dx = g["box_len_cm"] / N
    rs = (3 * 5e48 / (4 * np.pi * ALPHA_B * 1e-3 ** 2)) ** (1 / 3)
    trec = 1.0 / (ALPHA_B * 1e-3)
    r_if = rs * (1 - np.exp(-t_myr * MYR_S / trec)) ** (1 / 3) / dx
    i = np.arange(N) + 0.5
    r = np.sqrt(i[None, None, :] ** 2 + i[None, :, None] ** 2 + i[:, None, None] ** 2).reshape(-1)
    w = width_cells * N / 128.0
    x = x_in + (1.0 - x_in) / (1.0 + np.exp(-(r - r_if) / w))
    g["x_HI"] = x
    g["x_HII"] = (1.0 - x_in) - (1.0 - x_in) / (1.0 + np.exp(-(r - r_if) / w))
    g["r_if_cells"] = r_if
    return g


def lognormal_density(N: int, sigma_ln: float = 1.0, mean: float = 1e-2, seed: int = BASE_SEED,
                      dims=None) -> np.ndarray:
    """Log-normal medium from a P(k) ~ k^-3 Gaussian field, flattened x-fastest."""
    if dims is None:
        dims = (N, N, N)
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((nz, ny, nx))
    W = np.fft.rfftn(w)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** -1.5
    g = np.fft.irfftn(W * amp, s=(nz, ny, nx), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    e = np.exp(sigma_ln * g)
    n = mean * e / e.mean()
    return round_f32(n.reshape(-1))


def random_sources(dims, dx: float, nsrc: int, ndot_lo: float, ndot_hi: float, rng,
                   e_lo: float = 13.6, e_hi: float = 29.6):
    dims = np.asarray(dims)
    idx = np.stack([rng.integers(0, dims[i], nsrc) for i in range(3)], axis=1)
    pos = cell_centre_cm(idx, dx)
    ndot = np.exp(rng.uniform(np.log(ndot_lo), np.log(ndot_hi), nsrc))
    e = rng.uniform(e_lo, e_hi, nsrc)
    return pos, ndot, e, np.full(nsrc, SIGMA_HI)


def clumpy(N: int = 256, nsrc: int = 1000, seed: int = BASE_SEED + 2, box_kpc: float = 6.6) -> dict:
    """Clumpy multi-source medium (log-normal density, many sources)."""
    rng = np.random.default_rng(seed)
    box = box_cm(N, box_kpc)
    dx = box / N
    n = lognormal_density(N, seed=seed)
    pos, ndot, e, sg = random_sources((N, N, N), dx, nsrc, 1e48, 1e50, rng)
    return _grid(N, box, n, 1.0, pos, ndot, e, sg, alpha_B=ALPHA_B)


BATCH_SIDES = (32, 48, 64, 96, 128, 192)


def batch(n_inst: int = 64, seed: int = BASE_SEED + 3, box_kpc: float = 6.6,
          max_src: int = 256) -> list:
    """Independent instances of uneven size and source count."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        N = int(rng.choice(BATCH_SIDES))
        nsrc = int(rng.integers(1, max_src + 1))
        box = box_cm(N, box_kpc)
        n = lognormal_density(N, seed=seed * 1000 + i)
        pos, ndot, e, sg = random_sources((N, N, N), box / N, nsrc, 1e47, 1e50, rng)
        out.append(_grid(N, box, n, 1.0, pos, ndot, e, sg, alpha_B=ALPHA_B))
    return out


def request_stream(rate_hz: float = 200.0, duration_s: float = 60.0, seed: int = BASE_SEED + 4,
                   n_lo: int = 64, n_hi: int = 256, max_src: int = 500, max_steps: int = 20) -> list:
    """Poisson request arrivals: (arrival_s, N, nsrc, nsteps, seed) per request."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        cells = np.exp(rng.uniform(np.log(float(n_lo) ** 3), np.log(float(n_hi) ** 3)))
        N = int(round(cells ** (1.0 / 3.0)))
        out.append(dict(arrival_s=t, N=N, nsrc=int(rng.integers(1, max_src + 1)),
                        nsteps=int(rng.integers(1, max_steps + 1)),
                        seed=int(rng.integers(0, 2 ** 31))))
    return out


def request_grid(req: dict, box_kpc: float = 6.6) -> dict:
    """Materialise the grid of one request from the stream."""
    rng = np.random.default_rng(req["seed"])
    N = req["N"]
    box = box_cm(N, box_kpc)
    n = lognormal_density(N, seed=req["seed"])
    pos, ndot, e, sg = random_sources((N, N, N), box / N, req["nsrc"], 1e47, 1e50, rng)
    return _grid(N, box, n, 1.0, pos, ndot, e, sg, alpha_B=ALPHA_B)


E_ION_EV = (13.6, 24.6, 54.4)              # H I, He I, He II ionisation energies
SIGMA_TYPE = (6.3e-18, 7.43e-18, 1.58e-18)  # threshold cross sections of the three absorbers


def typed_clumpy(N: int = 128, nsrc: int = 30, seed: int = BASE_SEED + 6, box_kpc: float = 6.6) -> dict:
    """The clumpy medium with sources of the three photon types and helium
    absorbers; adds ``types`` and ``n_he`` (2, ncell) to the grid dict."""
    g = clumpy(N, nsrc, seed, box_kpc)
    rng = np.random.default_rng(seed + 1)
    types = np.arange(nsrc) % 3
    e_ion = np.asarray(E_ION_EV)[types]
    g["e_ph_eV"] = e_ion + rng.uniform(0.0, 16.0, nsrc)
    g["sigma_cm2"] = np.asarray(SIGMA_TYPE)[types]
    g["types"] = types
    n_he = 0.079 * g["n_H"]
    g["n_he"] = np.stack([round_f32(0.9 * n_he), round_f32(0.1 * n_he)])
    return g


def pulse_rate(t_s, L_max: float = 1e55, t0_s: float = 0.5 * MYR_S, A: float = 4.0):
    """Eq. "test12" (Application 5): L(t) = L_max exp[A (t_f / t0 - 1)] with
    t_f = 2 |t - t0 round(t / t0)|, a pulse of period t0 peaking at t0/2 + k t0."""
    t = np.asarray(t_s, dtype=np.float64)
    tf = 2.0 * np.abs(t - t0_s * np.round(t / t0_s))
    return L_max * np.exp(A * (tf / t0_s - 1.0))


def pulse(N: int = 128, box_kpc: float = 1000.0, n_H: float = 1e-4, x_HI: float = 1e-5,
          e_ph: float = 29.6) -> dict:
    """Application 5 (Sec. 9) medium on an N^3 grid: uniform, optically thin,
    one source at the domain corner with the pulse's initial rate; the caller
    sets the rate of every step from pulse_rate(t)."""
    g = _grid(N, box_cm(N, box_kpc), n_H, x_HI, [[0.0, 0.0, 0.0]], [float(pulse_rate(0.0))], [e_ph], [SIGMA_HI],
              alpha_B=ALPHA_B)
    g["dt_s"] = 0.05 * MYR_S
    g["light_cm"] = C_CM_S * g["dt_s"]
    return g
