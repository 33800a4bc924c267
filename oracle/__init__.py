"""FP64 CPU oracle for photon-conserving adaptive ray tracing (arXiv:1012.2865).

TEST INFRASTRUCTURE ONLY.  This package is the reference the CUDA path is
checked against; the library itself never imports it.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

The arithmetic lives in ``rt_oracle.c`` (plain C, FP64, compiled without FMA
contraction); this module only builds it and marshals numpy arrays:

* ``pix2vec`` / ``pix2ang`` / ``ang2pix`` -- HEALPix nested scheme (Sec. 2.1,
  Step 3a).
* ``ray_path`` -- cell sequence and segment lengths of one unsplit ray
  (Eq. "trace", Step 3d).
* ``trace`` -- Steps 1-5 of Sec. 3.1 for every source of a grid: k_ph and
  Gamma per cell (Eqs. "dtau", "flux", "kph", "gamma"), the photon budget,
  packages created per HEALPix level and a checksum of the created set.
* ``trace_roots`` -- the same pass for a range of root packages (the
  pass is their sum; used to share a trace among host threads).
* ``chem`` -- backward-Euler update of Eq. "dndt" (hydrogen only).
* ``trace(..., src_type=, n_he=)`` -- photon types (Sec. 3.2): H I, He I
  and He II ionising packages, each absorbed by its own species.
* ``Flight`` / ``trace(..., flight=, light_cm=)`` -- finite speed of light
  (Sec. 2.1, Step 3j): packages halt after travelling c dt_P in a trace and
  continue in the next one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

MAX_LEVEL = 14
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB = os.path.join(_HERE, "librt_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rt_oracle.c into librt_oracle.so (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint64
            p = ctypes.c_void_p
            lib.orc_pix2vec_nest.argtypes = [i, u64, p]
            lib.orc_pix2vec_nest.restype = None
            lib.orc_pix2ang_nest.argtypes = [i, u64, p, p]
            lib.orc_pix2ang_nest.restype = None
            lib.orc_ang2pix_nest.argtypes = [i, d, d]
            lib.orc_ang2pix_nest.restype = u64
            lib.orc_ray_path.argtypes = [p, p, p, d, i, p, p, p]
            lib.orc_ray_path.restype = i
            lib.orc_trace.argtypes = [p, d, p, p, i, p, p, p, p, i, d, d, i, p, p, p, p, p, p, i, i]
            lib.orc_trace.restype = i
            lib.orc_trace_fsl.argtypes = [p, d, p, p, i, p, p, p, p, i, d, d, i, p, p, p, p, p, p, i, i,
                                          i, p, ctypes.c_size_t, p, ctypes.c_size_t, p, p]
            lib.orc_trace_fsl.restype = i
            lib.orc_trace_mf.argtypes = [p, d, p, p, p, i, p, p, p, p, p, i, d, d, i, p, p, p, p, p, p, i, i,
                                         i, p, ctypes.c_size_t, p, ctypes.c_size_t, p, p]
            lib.orc_trace_mf.restype = i
            lib.orc_trace_roots.argtypes = [p, d, p, p, i, p, p, p, p, i, d, d, i, p, p, p, p, p, p, u64, u64]
            lib.orc_trace_roots.restype = i
            lib.orc_chem.argtypes = [ctypes.c_size_t, p, p, p, p, d, i, d]
            lib.orc_chem.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def pix2vec(level: int, pix) -> np.ndarray:
    """Unit vectors of nested pixel centres, shape (len(pix), 3)."""
    lib = _load()
    pix = np.atleast_1d(np.asarray(pix, dtype=np.uint64))
    out = np.empty((pix.size, 3), dtype=np.float64)
    v = np.empty(3, dtype=np.float64)
    for j, p in enumerate(pix):
        lib.orc_pix2vec_nest(int(level), int(p), _ptr(v))
        out[j] = v
    return out


def pix2ang(level: int, pix):
    """(z, phi) of nested pixel centres, phi in [0, 2 pi)."""
    lib = _load()
    pix = np.atleast_1d(np.asarray(pix, dtype=np.uint64))
    z = np.empty(pix.size)
    phi = np.empty(pix.size)
    zz = ctypes.c_double()
    pp = ctypes.c_double()
    for j, p in enumerate(pix):
        lib.orc_pix2ang_nest(int(level), int(p), ctypes.byref(zz), ctypes.byref(pp))
        z[j] = zz.value
        phi[j] = pp.value
    return z, phi


def ang2pix(level: int, z, phi) -> np.ndarray:
    lib = _load()
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
    out = np.empty(z.size, dtype=np.uint64)
    for j in range(z.size):
        out[j] = lib.orc_ang2pix_nest(int(level), float(z[j]), float(phi[j]))
    return out


def ray_path(dims, s, n, r0: float = 0.0, max_out: int = 100000):
    """Cells (k, 3), segment lengths and entry radii of one unsplit ray (cell units)."""
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    s = _f64(s)
    n = _f64(n)
    cells = np.empty((max_out, 3), dtype=np.int64)
    dr = np.empty(max_out)
    r = np.empty(max_out)
    k = lib.orc_ray_path(_ptr(dims), _ptr(s), _ptr(n), float(r0), int(max_out), _ptr(cells),
                         _ptr(dr), _ptr(r))
    return cells[:k].copy(), dr[:k].copy(), r[:k].copy()


# A package kept between traces (finite speed of light): the layout of
# orc_flight in rt_oracle.c.  r in cell units, P in photons/s, cell = the
# cell it halted in, age = its index into the next trace's halting radii.
FLIGHT_DTYPE = np.dtype([("src", "<u4"), ("level", "<u4"), ("pix", "<u8"), ("r", "<f8"), ("P", "<f8"),
                         ("tau", "<f8"), ("cell", "<i8", (3,)), ("age", "<u4"), ("pad", "<u4")])


class Flight:
    """Packages of one grid in flight between traces, and the halting radii.

    Sec. 2.1 (first halting condition) and Step 3j: a package travels c dt_P
    per radiative-transfer timestep and is then saved and continued in the
    next step, through the medium of that step.  Ages count the traces since
    a package's lineage was emitted; in a trace whose light travel is
    c dt_P (cell units) a package of age a halts at
        rlim[0] = c dt_P,   rlim[a] = rlim_previous[a - 1] + c dt_P,
    the distance light has travelled since its emission (reading R15).
    """

    def __init__(self):
        self.rlim = np.zeros(0)
        self.packages = np.zeros(0, dtype=FLIGHT_DTYPE)

    def advance(self, c_dt_cells: float) -> np.ndarray:
        """Halting radii of the next trace (one more age than before)."""
        prev = self.rlim
        new = np.empty(prev.size + 1)
        new[0] = c_dt_cells
        for a in range(1, new.size):
            new[a] = prev[a - 1] + c_dt_cells
        self.rlim = new
        return new


def trace(dims, box_len_cm: float, n_H, x_HI, pos_cm, ndot, e_ph_eV, sigma_cm2, *,
          level0: int = 1, phi_c: float = 5.1, f_term: float = 1e-10,
          max_level: int = MAX_LEVEL, fc: bool = False, src_offset: int = 0,
          flight: Flight = None, light_cm: float = 0.0, src_type=None, n_he=None) -> dict:
    """One radiative-transfer pass (Steps 1-5).  Cell index = i + nx*(j + ny*k).

    Returns dict(kph, gamma (per cell, s^-1 and erg/s), budget=[emitted,
    absorbed, escaped] (photons/s), counts[15], hashes[15], segments).

    With ``flight`` and ``light_cm`` = c dt_P > 0 (finite speed of light),
    the packages in ``flight`` continue alongside the sources' new packages,
    every package halts where it has travelled c dt_P since its emission, and ``flight`` afterwards holds the halted packages; the result
    adds ``resumed`` and ``halted`` (photons/s) and ``n_halted``.  With
    ``light_cm`` = 0 any packages in ``flight`` are dropped.

    Photon types (Sec. 3.2): ``src_type[s]`` in {0: H I, 1: He I, 2: He II}
    and ``n_he`` = (n_HeI, n_HeII) per cell; a package is absorbed by its
    type's species only.  The result then adds ``kph_types`` and
    ``gamma_types`` of shape (3, ncell); ``kph`` / ``gamma`` stay the H I
    rates.
    """
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    ncell = int(np.prod(dims.astype(np.int64)))
    n_H = _f64(n_H).reshape(-1)
    x_HI = _f64(x_HI).reshape(-1)
    assert n_H.size == ncell and x_HI.size == ncell
    pos = _f64(pos_cm).reshape(-1)
    ndot = _f64(ndot).reshape(-1)
    nsrc = ndot.size
    e = _f64(e_ph_eV).reshape(-1)
    sg = _f64(sigma_cm2).reshape(-1)
    assert pos.size == 3 * nsrc and e.size == nsrc and sg.size == nsrc
    nt = 3 if n_he is not None else 1
    he = _f64(n_he).reshape(-1) if n_he is not None else np.zeros(1)
    assert n_he is None or he.size == 2 * ncell
    st = np.ascontiguousarray(src_type, dtype=np.int32).reshape(-1) if src_type is not None else None
    assert st is None or st.size == nsrc
    kph_all = np.empty(nt * ncell)
    gamma_all = np.empty(nt * ncell)
    budget = np.empty(5)
    counts = np.zeros(MAX_LEVEL + 1, dtype=np.uint64)
    hashes = np.zeros(MAX_LEVEL + 1, dtype=np.uint64)
    seg = np.zeros(1, dtype=np.uint64)
    finite = flight is not None and light_cm > 0
    if flight is not None and not finite:
        flight.rlim = np.zeros(0)
        flight.packages = np.zeros(0, dtype=FLIGHT_DTYPE)
    rlim = np.ascontiguousarray(flight.advance(float(light_cm) / (float(box_len_cm) / int(dims[0])))) \
        if finite else np.zeros(1)
    pin = np.ascontiguousarray(flight.packages if finite else np.zeros(0, dtype=FLIGHT_DTYPE))
    cap = max(1024, 4 * pin.size)
    n_out = ctypes.c_size_t(0)
    while True:
        out = np.zeros(cap, dtype=FLIGHT_DTYPE)
        rc = lib.orc_trace_mf(_ptr(dims), float(box_len_cm), _ptr(n_H), _ptr(x_HI),
                              _ptr(he) if n_he is not None else None, int(nsrc), _ptr(pos),
                              _ptr(ndot), _ptr(e), _ptr(sg), _ptr(st) if st is not None else None,
                              int(level0), float(phi_c), float(f_term),
                              int(max_level), _ptr(kph_all), _ptr(gamma_all), _ptr(budget), _ptr(counts),
                              _ptr(hashes), _ptr(seg), 1 if fc else 0, int(src_offset),
                              int(rlim.size) if finite else 0, _ptr(rlim), ctypes.c_size_t(pin.size),
                              _ptr(pin), ctypes.c_size_t(cap), _ptr(out), ctypes.byref(n_out))
        if rc == -2:
            cap = int(n_out.value)
            continue
        break
    if rc != 0:
        raise ValueError("oracle trace rejected its arguments")
    res = dict(kph=kph_all[:ncell].copy(), gamma=gamma_all[:ncell].copy(), budget=budget[:3].copy(),
               counts=counts, hashes=hashes, segments=int(seg[0]))
    if n_he is not None:
        res.update(kph_types=kph_all.reshape(3, ncell), gamma_types=gamma_all.reshape(3, ncell))
    if finite:
        flight.packages = out[:n_out.value].copy()
        res.update(resumed=float(budget[3]), halted=float(budget[4]), n_halted=int(n_out.value))
    return res


def trace_roots(dims, box_len_cm: float, n_H, x_HI, pos_cm, ndot, e_ph_eV, sigma_cm2, root_first: int,
                root_count: int, *, level0: int = 1, phi_c: float = 5.1, f_term: float = 1e-10,
                max_level: int = MAX_LEVEL) -> dict:
    """``trace`` restricted to the root packages src * 12 * 4^level0 + pixel in
    [root_first, root_first + root_count) (H I photons, infinite speed of
    light).  Disjoint ranges covering every root sum to the whole pass, so
    host threads can share one trace (the C call releases the GIL)."""
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    ncell = int(np.prod(dims.astype(np.int64)))
    n_H = _f64(n_H).reshape(-1)
    x_HI = _f64(x_HI).reshape(-1)
    assert n_H.size == ncell and x_HI.size == ncell
    pos = _f64(pos_cm).reshape(-1)
    ndot = _f64(ndot).reshape(-1)
    nsrc = ndot.size
    e = _f64(e_ph_eV).reshape(-1)
    sg = _f64(sigma_cm2).reshape(-1)
    assert pos.size == 3 * nsrc and e.size == nsrc and sg.size == nsrc
    kph = np.empty(ncell)
    gamma = np.empty(ncell)
    budget = np.empty(3)
    counts = np.zeros(MAX_LEVEL + 1, dtype=np.uint64)
    hashes = np.zeros(MAX_LEVEL + 1, dtype=np.uint64)
    seg = np.zeros(1, dtype=np.uint64)
    rc = lib.orc_trace_roots(_ptr(dims), float(box_len_cm), _ptr(n_H), _ptr(x_HI), int(nsrc), _ptr(pos), _ptr(ndot),
                             _ptr(e), _ptr(sg), int(level0), float(phi_c), float(f_term), int(max_level), _ptr(kph),
                             _ptr(gamma), _ptr(budget), _ptr(counts), _ptr(hashes), _ptr(seg), int(root_first),
                             int(root_count))
    if rc != 0:
        raise ValueError("oracle trace rejected its arguments")
    return dict(kph=kph, gamma=gamma, budget=budget, counts=counts, hashes=hashes, segments=int(seg[0]))


def chem(n_H, x_HI, x_HII, kph, dt_s: float, nsub: int, alpha_B: float):
    """Backward-Euler update of Eq. "dndt"; returns new (x_HI, x_HII) arrays."""
    lib = _load()
    n_H = _f64(n_H).reshape(-1)
    x = _f64(x_HI).reshape(-1).copy()
    z = _f64(x_HII).reshape(-1).copy()
    k = _f64(kph).reshape(-1)
    assert n_H.size == x.size == z.size == k.size
    lib.orc_chem(ctypes.c_size_t(x.size), _ptr(n_H), _ptr(x), _ptr(z), _ptr(k), float(dt_s),
                 int(nsub), float(alpha_B))
    return x, z
