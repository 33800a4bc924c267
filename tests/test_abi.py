"""The C-ABI library builds for sm_103a, loads, and exports every symbol rt.h declares.

No compute call is made here (no GPU on the CPU runners)."""
import ctypes

from paper_1012_2865_gb300 import build, native


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    L = ctypes.CDLL(path)
    syms = native.header_symbols()
    assert len(syms) >= 14
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    for core in ("rt_create_grid", "rt_add_sources", "rt_trace", "rt_chem_update", "rt_get_rates"):
        assert core in syms


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the rt.h structs have the C compiler's sizes and offsets."""
    import os
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "rt.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(rt_grid_desc), offsetof(rt_grid_desc, box_len_cm),
         offsetof(rt_grid_desc, n_H), offsetof(rt_grid_desc, x_HII));
  printf("%zu %zu %zu %zu\n", sizeof(rt_trace_params), offsetof(rt_trace_params, phi_c),
         offsetof(rt_trace_params, queue_capacity), offsetof(rt_trace_params, segs_per_iter));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(rt_budget), offsetof(rt_budget, counts),
         offsetof(rt_budget, segments), offsetof(rt_budget, status), offsetof(rt_budget, passes),
         offsetof(rt_budget, n_halted));
  printf("%zu %zu\n", sizeof(rt_trace_params), offsetof(rt_trace_params, light_cm));
  printf("%zu %zu %zu\n", sizeof(rt_flight), offsetof(rt_flight, src), offsetof(rt_flight, cell));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(build.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                             check=True).stdout.strip().splitlines()]
    D, T, B = native.rt_grid_desc, native.rt_trace_params, native.rt_budget
    assert got[0] == [ctypes.sizeof(D), D.box_len_cm.offset, D.n_H.offset, D.x_HII.offset]
    assert got[1] == [ctypes.sizeof(T), T.phi_c.offset, T.queue_capacity.offset, T.segs_per_iter.offset]
    assert got[2] == [ctypes.sizeof(B), B.counts.offset, B.segments.offset, B.status.offset, B.passes.offset,
                      B.n_halted.offset]
    assert got[3] == [ctypes.sizeof(T), T.light_cm.offset]
    F = native.rt_flight
    assert got[4] == [ctypes.sizeof(F), F.src.offset, F.cell.offset]
    assert native.FLIGHT_DTYPE.itemsize == ctypes.sizeof(F)


def test_error_message_without_gpu_is_reported_not_raised_from_c():
    L = native.lib()
    h = ctypes.c_void_p()
    rc = L.rt_ctx_create(-1, ctypes.byref(h))
    assert rc != 0
    assert len(L.rt_get_last_error()) > 0


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built library every call raises: there is no CPU fallback."""
    import pytest
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB", native.LIB + ".absent")
    with pytest.raises(RuntimeError, match="no fallback"):
        native.lib()
    with pytest.raises(RuntimeError):
        native.rt_ctx_create(0)


def test_dims_query_rejects_a_null_grid():
    L = native.lib()
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.rt_get_dims(None, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == native.RT_ERR_INVALID_ARG
