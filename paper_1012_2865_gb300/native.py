"""ctypes binding of the C ABI in include/rt.h (argument marshalling only).

Every computation happens in librt_gb300.so's CUDA kernels.  Loading fails
loudly when the library has not been built; there is no fallback.

Buffers may be numpy arrays (host memory) or torch CUDA tensors (device
memory); torch is imported only when a tensor is passed.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB, ROOT

RT_OK = 0
RT_ERR_INVALID_ARG = 1
RT_ERR_OOM = 2
RT_ERR_CUDA = 3
RT_ERR_QUEUE_OVERFLOW = 4
RT_ERR_LEVEL_OVERFLOW = 5
RT_ERR_TIMEOUT = 6
RT_ERR_STATE = 7
RT_FP64 = 0
RT_FP32_MIXED = 1
RT_MEM_HOST = 0
RT_MEM_DEVICE = 1
RT_DTYPE_F64 = 0
RT_DTYPE_F32 = 1
RT_MAX_LEVEL = 14
RT_TRACE_CHECKSUMS = 1
RT_TRACE_FC = 2
RT_TRACE_SELFTEST_STALL = 4
NLEV = RT_MAX_LEVEL + 1

PRECISIONS = {"fp64": RT_FP64, "fp32_mixed": RT_FP32_MIXED, "mixed": RT_FP32_MIXED}


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


class rt_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("box_len_cm", ctypes.c_double), ("precision", ctypes.c_int),
                ("mem_kind", ctypes.c_int), ("n_H", ctypes.c_void_p), ("x_HI", ctypes.c_void_p),
                ("x_HII", ctypes.c_void_p)]


class rt_trace_params(ctypes.Structure):
    _fields_ = [("level0", ctypes.c_int), ("phi_c", ctypes.c_double), ("f_term", ctypes.c_double),
                ("max_level", ctypes.c_int), ("queue_capacity", ctypes.c_int64),
                ("timeout_s", ctypes.c_double), ("blocks_per_sm", ctypes.c_int),
                ("segs_per_iter", ctypes.c_int), ("flags", ctypes.c_int), ("passes", ctypes.c_int),
                ("light_cm", ctypes.c_double)]


class rt_budget(ctypes.Structure):
    _fields_ = [("emitted", ctypes.c_double), ("absorbed", ctypes.c_double),
                ("escaped", ctypes.c_double), ("counts", ctypes.c_uint64 * NLEV),
                ("hashes", ctypes.c_uint64 * NLEV), ("segments", ctypes.c_uint64),
                ("fallbacks", ctypes.c_uint64), ("fallbacks_tau", ctypes.c_uint64),
                ("queue_pushed", ctypes.c_uint64),
                ("status", ctypes.c_int), ("kernel_ms", ctypes.c_float),
                ("queue_peak", ctypes.c_uint64), ("passes", ctypes.c_int),
                ("resumed", ctypes.c_double), ("halted", ctypes.c_double),
                ("n_resumed", ctypes.c_uint64), ("n_halted", ctypes.c_uint64)]


class rt_flight(ctypes.Structure):
    _fields_ = [("r_cm", ctypes.c_double), ("P", ctypes.c_double), ("tau", ctypes.c_double),
                ("src", ctypes.c_int32), ("level", ctypes.c_int32), ("pix", ctypes.c_uint32),
                ("age", ctypes.c_uint32), ("cell", ctypes.c_int32 * 3), ("pad", ctypes.c_int32)]


# numpy view of an rt_flight array
FLIGHT_DTYPE = np.dtype([("r_cm", "<f8"), ("P", "<f8"), ("tau", "<f8"), ("src", "<i4"), ("level", "<i4"),
                         ("pix", "<u4"), ("age", "<u4"), ("cell", "<i4", (3,)), ("pad", "<i4")])


class rt_noalloc_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("box_len_cm", ctypes.c_double), ("n_HI", ctypes.c_void_p), ("n_H", ctypes.c_void_p),
                ("x_HI", ctypes.c_void_p), ("kph", ctypes.c_void_p), ("gamma", ctypes.c_void_p)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1012_2865_gb300.build.build()"
                               " (the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "rt_ctx_create": ([i, ctypes.POINTER(vp)], i),
            "rt_ctx_destroy": ([vp], i),
            "rt_create_grid": ([vp, ctypes.POINTER(rt_grid_desc), vp, ctypes.POINTER(vp)], i),
            "rt_grid_destroy": ([vp], i),
            "rt_add_sources": ([vp, i, vp, vp, vp, vp], i),
            "rt_clear_sources": ([vp], i),
            "rt_trace": ([vp, ctypes.POINTER(rt_trace_params), ctypes.POINTER(rt_budget)], i),
            "rt_get_budget": ([vp, ctypes.POINTER(rt_budget)], i),
            "rt_chem_update": ([vp, d, i, d], i),
            "rt_get_rates": ([vp, vp, vp, vp, i, i], i),
            "rt_set_state": ([vp, vp, vp, vp, i], i),
            "rt_set_state_async": ([vp, vp, vp, vp, i], i),
            "rt_get_rates_async": ([vp, vp, vp, vp, i, i], i),
            "rt_wait_rates": ([vp], i),
            "rt_get_ionised": ([vp, vp, i, i], i),
            "rt_set_rates": ([vp, vp, vp, i, i], i),
            "rt_timestep": ([vp, d, d, d, d, d, d, ctypes.POINTER(d)], i),
            "rt_set_source_offset": ([vp, i], i),
            "rt_set_source_rates": ([vp, i, vp], i),
            "rt_set_source_types": ([vp, i, vp], i),
            "rt_set_absorbers": ([vp, vp, vp, i], i),
            "rt_get_rates_typed": ([vp, i, vp, vp, i, i], i),
            "rt_get_in_flight": ([vp, vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)], i),
            "rt_synchronize": ([vp], i),
            "rt_get_dims": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "rt_selfcheck_directions": ([vp, i, ctypes.POINTER(d), ctypes.POINTER(d)], i),
            "rt_kernel_launches": ([], ctypes.c_uint64),
            "rt_get_last_error": ([], ctypes.c_char_p),
            "rt_batch_create": ([vp, vp, ctypes.POINTER(vp)], i),
            "rt_batch_destroy": ([vp], i),
            "rt_batch_add": ([vp, vp, ctypes.POINTER(i)], i),
            "rt_batch_remove": ([vp, i], i),
            "rt_batch_size": ([vp], i),
            "rt_batch_trace": ([vp, ctypes.POINTER(rt_trace_params), i], i),
            "rt_batch_chem": ([vp, d, i, d], i),
            "rt_batch_step": ([vp, ctypes.POINTER(rt_trace_params), d, i, d, i], i),
            "rt_batch_get_budget": ([vp, i, ctypes.POINTER(rt_budget)], i),
            "rt_batch_autotune": ([vp, ctypes.POINTER(rt_trace_params)], i),
            "rt_trace_noalloc": ([ctypes.POINTER(rt_noalloc_grid), i, vp, vp, vp, vp,
                                  ctypes.POINTER(rt_trace_params), vp, ctypes.POINTER(rt_budget)], i),
            "rt_noalloc_last_error": ([], ctypes.c_char_p),
            "rt_probe_red": ([i, i, ctypes.c_uint64, ctypes.POINTER(d)], i),
            "rt_probe_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_symbols() -> list:
    """Function names declared in include/rt.h."""
    with open(os.path.join(ROOT, "include", "rt.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rt_[a-z_]+)\s*\(",
                                 text, flags=re.M)))


def check(code):
    if code != RT_OK:
        raise RtError(code, lib().rt_get_last_error().decode(errors="replace"))


_TORCH_DTYPE = {np.dtype(np.float64): "torch.float64", np.dtype(np.float32): "torch.float32"}


def _buf(a, dtype=np.float64, n=None):
    """(pointer, mem_kind, keepalive) for a numpy array or a torch tensor.

    A host array is converted to a contiguous array of `dtype`; a CUDA tensor
    is passed as it is and must already have that element type and be
    contiguous.  With `n` given, the element count must be n: the library
    reads n elements through the pointer."""
    if a is None:
        return None, RT_MEM_HOST, None
    if type(a).__module__.startswith("torch"):
        if a.is_cuda:
            want = _TORCH_DTYPE[np.dtype(dtype)]
            if str(a.dtype) != want:
                raise TypeError(f"device array of {a.dtype}; expected {want}")
            if not a.is_contiguous():
                raise ValueError("device array is not contiguous")
            if n is not None and a.numel() != n:
                raise ValueError(f"device array of {a.numel()} elements; expected {n}")
            return a.data_ptr(), RT_MEM_DEVICE, a
        a = a.numpy()
    arr = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
    if n is not None and arr.size != n:
        raise ValueError(f"array of {arr.size} elements; expected {n}")
    return arr.ctypes.data, RT_MEM_HOST, arr


def rt_get_dims(grid) -> tuple:
    nx, ny, nz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().rt_get_dims(grid, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz)))
    return nx.value, ny.value, nz.value


def _ncell(grid) -> int:
    nx, ny, nz = rt_get_dims(grid)
    return nx * ny * nz


def rt_ctx_create(device: int = 0):
    h = ctypes.c_void_p()
    check(lib().rt_ctx_create(int(device), ctypes.byref(h)))
    return h


def rt_ctx_destroy(ctx):
    check(lib().rt_ctx_destroy(ctx))


def rt_create_grid(ctx, dims, box_len_cm, n_H, x_HI, x_HII=None, precision="fp64", stream=None):
    nx, ny, nz = (int(v) for v in dims)
    n = nx * ny * nz if min(nx, ny, nz) > 0 else None  # the library rejects empty dims itself
    pn, kn, kn_ = _buf(n_H, n=n)
    px, kx, kx_ = _buf(x_HI, n=n)
    pz, kz, kz_ = _buf(x_HII, n=n)
    if len({k for k, p in ((kn, pn), (kx, px), (kz, pz)) if p is not None}) > 1:
        raise ValueError("n_H, x_HI, x_HII must all live on the host or all on the device")
    d = rt_grid_desc(nx, ny, nz, float(box_len_cm), PRECISIONS[precision] if isinstance(precision, str)
                     else int(precision), kn, pn, px, pz)
    h = ctypes.c_void_p()
    check(lib().rt_create_grid(ctx, ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def rt_grid_destroy(grid):
    check(lib().rt_grid_destroy(grid))


def rt_add_sources(grid, pos_cm, ndot, e_ph_eV, sigma_cm2):
    pos = np.ascontiguousarray(pos_cm, dtype=np.float64).reshape(-1)
    nd = np.ascontiguousarray(ndot, dtype=np.float64).reshape(-1)
    e = np.ascontiguousarray(e_ph_eV, dtype=np.float64).reshape(-1)
    s = np.ascontiguousarray(sigma_cm2, dtype=np.float64).reshape(-1)
    n = nd.size
    if pos.size != 3 * n or e.size != n or s.size != n:
        raise ValueError("source arrays disagree in length")
    check(lib().rt_add_sources(grid, n, pos.ctypes.data, nd.ctypes.data, e.ctypes.data, s.ctypes.data))


def rt_clear_sources(grid):
    check(lib().rt_clear_sources(grid))


def trace_params(level0=1, phi_c=5.1, f_term=1e-10, max_level=RT_MAX_LEVEL, queue_capacity=0,
                 timeout_s=2.0, blocks_per_sm=0, segs_per_iter=0, checksums=False,
                 passes=0, fc=False, light_cm=0.0, selftest_stall=False) -> rt_trace_params:
    flags = (RT_TRACE_CHECKSUMS if checksums else 0) | (RT_TRACE_FC if fc else 0) | \
        (RT_TRACE_SELFTEST_STALL if selftest_stall else 0)
    return rt_trace_params(int(level0), float(phi_c), float(f_term), int(max_level),
                           int(queue_capacity), float(timeout_s), int(blocks_per_sm),
                           int(segs_per_iter), flags, int(passes), float(light_cm))


def budget_dict(b: rt_budget) -> dict:
    return dict(emitted=b.emitted, absorbed=b.absorbed, escaped=b.escaped,
                counts=np.array(b.counts[:], dtype=np.uint64),
                hashes=np.array(b.hashes[:], dtype=np.uint64), segments=int(b.segments),
                fallbacks=int(b.fallbacks), fallbacks_tau=int(b.fallbacks_tau),
                queue_pushed=int(b.queue_pushed), queue_peak=int(b.queue_peak), passes=int(b.passes),
                status=int(b.status),
                kernel_ms=float(b.kernel_ms), resumed=float(b.resumed), halted=float(b.halted),
                n_resumed=int(b.n_resumed), n_halted=int(b.n_halted))


def rt_trace(grid, params: rt_trace_params, sync: bool = True):
    if sync:
        b = rt_budget()
        check(lib().rt_trace(grid, ctypes.byref(params), ctypes.byref(b)))
        return budget_dict(b)
    check(lib().rt_trace(grid, ctypes.byref(params), None))
    return None


def rt_get_budget(grid) -> dict:
    b = rt_budget()
    check(lib().rt_get_budget(grid, ctypes.byref(b)))
    return budget_dict(b)


def rt_set_state(grid, x_HI, x_HII=None, n_H=None):
    n = _ncell(grid)
    px, kx, kx_ = _buf(x_HI, n=n)
    pz, kz, kz_ = _buf(x_HII, n=n)
    pn, kn, kn_ = _buf(n_H, n=n)
    if len({k for k, p in ((kn, pn), (kx, px), (kz, pz)) if p is not None}) > 1:
        raise ValueError("n_H, x_HI, x_HII must all live on the host or all on the device")
    check(lib().rt_set_state(grid, pn, px, pz, kx))


def _in_place(a, ptr) -> bool:
    """True when the pointer handed to the library is the caller's own buffer
    (not a converted copy that would be gone before a deferred copy runs)."""
    if a is None:
        return True
    own = a.data_ptr() if type(a).__module__.startswith("torch") else np.asarray(a).ctypes.data
    return own == ptr


def rt_set_state_async(grid, x_HI, x_HII=None, n_H=None):
    """Enqueue a new gas state (host arrays best pinned; they must stay unchanged
    until rt_synchronize).  A rejected state is reported by a later call."""
    n = _ncell(grid)
    px, kx, kx_ = _buf(x_HI, n=n)
    pz, kz, kz_ = _buf(x_HII, n=n)
    pn, kn, kn_ = _buf(n_H, n=n)
    if len({k for k, p in ((kn, pn), (kx, px), (kz, pz)) if p is not None}) > 1:
        raise ValueError("n_H, x_HI, x_HII must all live on the host or all on the device")
    if kx == RT_MEM_HOST and not all(_in_place(a, p) for a, p in ((x_HI, px), (x_HII, pz), (n_H, pn))):
        raise ValueError("host arrays for rt_set_state_async must be contiguous float64 (they are read later)")
    check(lib().rt_set_state_async(grid, pn, px, pz, kx))


def rt_get_rates_async(grid, kph=None, gamma=None, x_HI=None, dtype=RT_DTYPE_F64):
    """Enqueue copies of k_ph, Gamma and x_HI into caller buffers (all numpy
    arrays, best pinned, or all CUDA tensors) of element type dtype; complete
    after rt_wait_rates / rt_synchronize."""
    n = _ncell(grid)
    want = np.float64 if dtype == RT_DTYPE_F64 else np.float32
    bufs = [(None, None, None) if a is None else _buf(a, dtype=want, n=n) for a in (kph, gamma, x_HI)]
    kinds = {b[1] for b in bufs if b[0] is not None}
    if len(kinds) > 1:
        raise ValueError("the output buffers must all live on the host or all on the device")
    for a, b in zip((kph, gamma, x_HI), bufs):
        if b[1] == RT_MEM_HOST and not _in_place(a, b[0]):
            raise ValueError("host output buffers for rt_get_rates_async must be contiguous arrays of the dtype")
    kind = kinds.pop() if kinds else RT_MEM_HOST
    check(lib().rt_get_rates_async(grid, bufs[0][0], bufs[1][0], bufs[2][0], int(dtype), kind))


def rt_wait_rates(grid):
    check(lib().rt_wait_rates(grid))


def rt_set_source_offset(grid, first: int):
    check(lib().rt_set_source_offset(grid, int(first)))


def rt_set_source_rates(grid, ndot):
    nd = np.ascontiguousarray(ndot, dtype=np.float64).reshape(-1)
    check(lib().rt_set_source_rates(grid, nd.size, nd.ctypes.data))


def rt_set_source_types(grid, types):
    t = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    check(lib().rt_set_source_types(grid, t.size, t.ctypes.data))


def rt_set_absorbers(grid, n_HeI, n_HeII):
    """Helium absorber densities: host arrays or CUDA tensors (float64)."""
    n = _ncell(grid)
    p1, k1, keep1 = _buf(n_HeI, n=n)
    p2, k2, keep2 = _buf(n_HeII, n=n)
    if k1 != k2:
        raise ValueError("n_HeI and n_HeII must both live on the host or both on the device")
    check(lib().rt_set_absorbers(grid, p1, p2, k1))


def _check_ncell(grid, ncell):
    """The library writes the grid's number of cells: the caller's count must be it."""
    n = _ncell(grid)
    if int(ncell) != n:
        raise ValueError(f"ncell = {ncell}; the grid has {n} cells")
    return n


def rt_get_rates_typed(grid, ncell, ptype, dtype=RT_DTYPE_F64, where="host"):
    ncell = _check_ncell(grid, ncell)
    outs = {k: _out(ncell, dtype, where) for k in ("kph", "gamma")}
    mk = RT_MEM_DEVICE if where == "device" else RT_MEM_HOST
    ptr = {k: (v.data_ptr() if where == "device" else v.ctypes.data) for k, v in outs.items()}
    check(lib().rt_get_rates_typed(grid, int(ptype), ptr["kph"], ptr["gamma"], int(dtype), mk))
    return outs


def rt_get_in_flight(grid) -> np.ndarray:
    """Packages in flight after the last trace, as a FLIGHT_DTYPE array."""
    n = ctypes.c_uint64()
    check(lib().rt_get_in_flight(grid, None, 0, ctypes.byref(n)))
    out = np.zeros(int(n.value), dtype=FLIGHT_DTYPE)
    if out.size:
        check(lib().rt_get_in_flight(grid, out.ctypes.data, out.size, ctypes.byref(n)))
    return out


def rt_set_rates(grid, kph, gamma):
    """Install k_ph and Gamma: host arrays (sent as FP64) or CUDA tensors of
    one dtype (float32 or float64)."""
    n = _ncell(grid)
    dev = type(kph).__module__.startswith("torch") and kph.is_cuda
    if dev:
        if not (type(gamma).__module__.startswith("torch") and gamma.is_cuda and kph.dtype == gamma.dtype):
            raise TypeError("kph and gamma: CUDA tensors of one dtype")
        dt = RT_DTYPE_F64 if str(kph.dtype) == "torch.float64" else RT_DTYPE_F32
    else:
        dt = RT_DTYPE_F64
    npdt = np.float64 if dt == RT_DTYPE_F64 else np.float32
    pk, kk, keep_k = _buf(kph, npdt, n=n)
    pg, kg, keep_g = _buf(gamma, npdt, n=n)
    if kk != kg:
        raise ValueError("kph and gamma must both live on the host or both on the device")
    check(lib().rt_set_rates(grid, pk, pg, dt, kk))


def rt_timestep(grid, eps_ion=0.05, alpha_B=2.59e-13, sigma_front=6.3e-18, tau_front=0.5, dt_max=float("inf"),
                dt_prev=0.0) -> float:
    out = ctypes.c_double()
    check(lib().rt_timestep(grid, float(eps_ion), float(alpha_B), float(sigma_front), float(tau_front),
                            float(dt_max), float(dt_prev), ctypes.byref(out)))
    return out.value


def rt_chem_update(grid, dt_s, nsub, alpha_B):
    check(lib().rt_chem_update(grid, float(dt_s), int(nsub), float(alpha_B)))


def _out(n, dtype, where):
    if where == "device":
        import torch
        return torch.empty(n, dtype=torch.float64 if dtype == RT_DTYPE_F64 else torch.float32,
                           device="cuda")
    return np.empty(n, dtype=np.float64 if dtype == RT_DTYPE_F64 else np.float32)


def rt_get_rates(grid, ncell, dtype=RT_DTYPE_F64, where="host", want=("kph", "gamma", "x_HI")):
    ncell = _check_ncell(grid, ncell)
    outs = {k: _out(ncell, dtype, where) if k in want else None for k in ("kph", "gamma", "x_HI")}
    mk = RT_MEM_DEVICE if where == "device" else RT_MEM_HOST
    ptr = {k: (None if v is None else (v.data_ptr() if where == "device" else v.ctypes.data))
           for k, v in outs.items()}
    check(lib().rt_get_rates(grid, ptr["kph"], ptr["gamma"], ptr["x_HI"], int(dtype), mk))
    return outs


def rt_get_ionised(grid, ncell, dtype=RT_DTYPE_F64, where="host"):
    ncell = _check_ncell(grid, ncell)
    out = _out(ncell, dtype, where)
    p = out.data_ptr() if where == "device" else out.ctypes.data
    check(lib().rt_get_ionised(grid, p, int(dtype), RT_MEM_DEVICE if where == "device" else RT_MEM_HOST))
    return out


def rt_selfcheck_directions(ctx, level: int):
    e = ctypes.c_double()
    b = ctypes.c_double()
    check(lib().rt_selfcheck_directions(ctx, int(level), ctypes.byref(e), ctypes.byref(b)))
    return e.value, b.value


def rt_synchronize(grid):
    check(lib().rt_synchronize(grid))


def rt_probe_red(device: int, dtype=RT_DTYPE_F32, words: int = 1 << 21) -> float:
    """Atomic reductions per second into an array of `words` elements (measurement aid)."""
    r = ctypes.c_double()
    code = lib().rt_probe_red(int(device), int(dtype), int(words), ctypes.byref(r))
    if code != RT_OK:
        raise RtError(code, lib().rt_probe_last_error().decode(errors="replace"))
    return r.value


def rt_kernel_launches() -> int:
    return int(lib().rt_kernel_launches())


def rt_get_last_error() -> str:
    return lib().rt_get_last_error().decode(errors="replace")


class Grid:
    """Convenience owner of one grid handle (marshalling only)."""

    def __init__(self, ctx, g: dict, precision="fp64", stream=None):
        self.dims = tuple(g["dims"])
        self.ncell = int(np.prod(self.dims))
        self.h = rt_create_grid(ctx, self.dims, g["box_len_cm"], g["n_H"], g["x_HI"],
                                g.get("x_HII"), precision, stream)
        if len(g["ndot"]):
            try:
                rt_add_sources(self.h, g["pos_cm"], g["ndot"], g["e_ph_eV"], g["sigma_cm2"])
            except (RtError, ValueError):
                rt_grid_destroy(self.h)  # a grid whose sources were refused is not kept
                self.h = None
                raise

    def trace(self, sync=True, **kw):
        return rt_trace(self.h, trace_params(**kw), sync=sync)

    def chem(self, dt_s, nsub=10, alpha_B=2.59e-13):
        rt_chem_update(self.h, dt_s, nsub, alpha_B)

    def set_source_rates(self, ndot):
        rt_set_source_rates(self.h, ndot)

    def in_flight(self) -> np.ndarray:
        return rt_get_in_flight(self.h)

    def set_source_types(self, types):
        rt_set_source_types(self.h, types)

    def set_absorbers(self, n_HeI, n_HeII):
        rt_set_absorbers(self.h, n_HeI, n_HeII)

    def rates_typed(self, ptype, dtype=RT_DTYPE_F64, where="host"):
        return rt_get_rates_typed(self.h, self.ncell, ptype, dtype, where)

    def rates(self, dtype=RT_DTYPE_F64, where="host"):
        return rt_get_rates(self.h, self.ncell, dtype, where)

    def x_HII(self):
        return rt_get_ionised(self.h, self.ncell)

    def close(self):
        if self.h:
            rt_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_trace_noalloc(dims, box_len_cm, n_HI, n_H, x_HI, kph, gamma, pos_cm, ndot, e_ph_eV, sigma_cm2,
                     params: rt_trace_params, stream=None) -> dict:
    """Allocation-free trace; every grid array is a CUDA tensor of nx*ny*nz
    elements (n_HI, kph, gamma float32; n_H, x_HI float64)."""
    nx, ny, nz = (int(v) for v in dims)
    n = nx * ny * nz if min(nx, ny, nz) > 0 else None  # the library rejects empty dims itself
    ptr = []
    for a, dt in ((n_HI, np.float32), (n_H, np.float64), (x_HI, np.float64), (kph, np.float32),
                  (gamma, np.float32)):
        p, kind, _ = _buf(a, dt, n=n)
        if kind != RT_MEM_DEVICE:
            raise ValueError("rt_trace_noalloc: the grid arrays are CUDA tensors")
        ptr.append(p)
    g = rt_noalloc_grid(nx, ny, nz, float(box_len_cm), *ptr)
    pos = np.ascontiguousarray(pos_cm, dtype=np.float64).reshape(-1)
    nd = np.ascontiguousarray(ndot, dtype=np.float64).reshape(-1)
    e = np.ascontiguousarray(e_ph_eV, dtype=np.float64).reshape(-1)
    sg = np.ascontiguousarray(sigma_cm2, dtype=np.float64).reshape(-1)
    if pos.size != 3 * nd.size or e.size != nd.size or sg.size != nd.size:
        raise ValueError("source arrays disagree in length")
    b = rt_budget()
    code = lib().rt_trace_noalloc(ctypes.byref(g), nd.size, pos.ctypes.data, nd.ctypes.data, e.ctypes.data,
                                  sg.ctypes.data, ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                  ctypes.byref(b))
    if code != RT_OK:
        raise RtError(code, lib().rt_noalloc_last_error().decode(errors="replace"))
    return budget_dict(b)


def rt_batch_create(ctx, stream=None):
    h = ctypes.c_void_p()
    check(lib().rt_batch_create(ctx, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def rt_batch_destroy(batch):
    check(lib().rt_batch_destroy(batch))


def rt_batch_add(batch, grid) -> int:
    slot = ctypes.c_int()
    check(lib().rt_batch_add(batch, grid, ctypes.byref(slot)))
    return slot.value


def rt_batch_remove(batch, slot):
    check(lib().rt_batch_remove(batch, int(slot)))


def rt_batch_size(batch) -> int:
    return int(lib().rt_batch_size(batch))


def rt_batch_trace(batch, params: rt_trace_params, sync: bool = True):
    check(lib().rt_batch_trace(batch, ctypes.byref(params), 1 if sync else 0))


def rt_batch_chem(batch, dt_s, nsub, alpha_B):
    check(lib().rt_batch_chem(batch, float(dt_s), int(nsub), float(alpha_B)))


def rt_batch_step(batch, params: rt_trace_params, dt_s, nsub, alpha_B, nsteps):
    check(lib().rt_batch_step(batch, ctypes.byref(params), float(dt_s), int(nsub), float(alpha_B), int(nsteps)))


def rt_batch_get_budget(batch, slot) -> dict:
    b = rt_budget()
    check(lib().rt_batch_get_budget(batch, int(slot), ctypes.byref(b)))
    return budget_dict(b)


def rt_batch_autotune(batch, params: rt_trace_params) -> rt_trace_params:
    check(lib().rt_batch_autotune(batch, ctypes.byref(params)))
    return params


class Batch:
    """Convenience owner of one batch handle (marshalling only)."""

    def __init__(self, ctx, stream=None):
        self.h = rt_batch_create(ctx, stream)
        self.grids = {}

    def add(self, grid: "Grid") -> int:
        slot = rt_batch_add(self.h, grid.h)
        self.grids[slot] = grid
        return slot

    def remove(self, slot: int):
        rt_batch_remove(self.h, slot)
        self.grids.pop(slot, None)

    def trace(self, sync=True, **kw):
        rt_batch_trace(self.h, trace_params(**kw), sync)

    def chem(self, dt_s, nsub=10, alpha_B=2.59e-13):
        rt_batch_chem(self.h, dt_s, nsub, alpha_B)

    def step(self, nsteps, dt_s, nsub=10, alpha_B=2.59e-13, **kw):
        rt_batch_step(self.h, trace_params(**kw), dt_s, nsub, alpha_B, nsteps)

    def budget(self, slot) -> dict:
        return rt_batch_get_budget(self.h, slot)

    def close(self):
        if self.h:
            rt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
