"""The binding's argument checks, on the host with a stand-in for the
library: per-cell arrays must have the grid's number of cells, CUDA tensors
must already have the element type the call reads and be contiguous, and the
arrays of one call live in one kind of memory.  A failed check raises before
the library is called, so no kernel ever reads past a caller's buffer.
"""
import numpy as np
import pytest

from paper_1012_2865_gb300 import native


class FakeDtype:
    def __init__(self, name):
        self.name = name

    def __str__(self):
        return self.name

    def __eq__(self, other):
        return str(self) == str(other)

    def __hash__(self):
        return hash(self.name)


class FakeCudaTensor:
    """Quacks like a CUDA torch tensor (the binding checks the module name)."""

    def __init__(self, n, dtype="torch.float64", contiguous=True, ptr=0x7000):
        self.n, self.dtype, self.contig, self.ptr = n, FakeDtype(dtype), contiguous, ptr
        self.is_cuda = True

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.contig

    def data_ptr(self):
        return self.ptr


FakeCudaTensor.__module__ = "torch.fake"


class FakeLib:
    dims = (4, 5, 6)

    def __init__(self):
        self.calls = []

    def rt_get_last_error(self):
        return b"fake"

    def rt_get_dims(self, grid, nx, ny, nz):
        nx._obj.value, ny._obj.value, nz._obj.value = self.dims
        return native.RT_OK

    def rt_create_grid(self, ctx, pd, stream, ph):
        d = pd._obj
        self.calls.append(("create", d.nx, d.ny, d.nz, d.mem_kind))
        return native.RT_ERR_INVALID_ARG if min(d.nx, d.ny, d.nz) < 1 else native.RT_OK

    def rt_set_state(self, grid, pn, px, pz, kind):
        self.calls.append(("state", pn, px, pz, kind))
        return native.RT_OK

    def rt_set_absorbers(self, grid, p1, p2, kind):
        self.calls.append(("absorbers", p1, p2, kind))
        return native.RT_OK

    def rt_set_rates(self, grid, pk, pg, dt, kind):
        self.calls.append(("rates", pk, pg, dt, kind))
        return native.RT_OK

    def rt_trace_noalloc(self, pg, nsrc, pos, nd, e, sg, params, stream, pb):
        g = pg._obj
        self.calls.append(("noalloc", g.n_HI, g.n_H, g.x_HI, g.kph, g.gamma, nsrc))
        return native.RT_OK

    def rt_noalloc_last_error(self):
        return b"fake"


@pytest.fixture
def fake(monkeypatch):
    L = FakeLib()
    monkeypatch.setattr(native, "_lib", L)
    return L


N = 4 * 5 * 6


def test_create_grid_checks_sizes(fake):
    native.rt_create_grid(None, (4, 5, 6), 1.0, np.ones(N), np.zeros((6, 5, 4)))
    assert fake.calls[-1] == ("create", 4, 5, 6, native.RT_MEM_HOST)
    with pytest.raises(ValueError):
        native.rt_create_grid(None, (4, 5, 6), 1.0, np.ones(N - 1), np.zeros(N))
    with pytest.raises(ValueError):
        native.rt_create_grid(None, (4, 5, 6), 1.0, np.ones(N), np.zeros(N), x_HII=np.zeros(N + 1))
    # empty dimensions are the library's to reject (RT_ERR_INVALID_ARG)
    with pytest.raises(native.RtError) as e:
        native.rt_create_grid(None, (4, 4, 0), 1.0, np.ones(64), np.zeros(64))
    assert e.value.code == native.RT_ERR_INVALID_ARG


def test_set_state_checks_device_arrays(fake):
    native.rt_set_state("g", FakeCudaTensor(N), FakeCudaTensor(N, ptr=0x8000))
    assert fake.calls[-1] == ("state", None, 0x7000, 0x8000, native.RT_MEM_DEVICE)
    with pytest.raises(TypeError):
        native.rt_set_state("g", FakeCudaTensor(N, dtype="torch.float32"))
    with pytest.raises(ValueError):
        native.rt_set_state("g", FakeCudaTensor(N, contiguous=False))
    with pytest.raises(ValueError):
        native.rt_set_state("g", FakeCudaTensor(N // 2))
    with pytest.raises(ValueError):
        native.rt_set_state("g", FakeCudaTensor(N), x_HII=np.zeros(N))  # host and device mixed
    n_calls = len(fake.calls)
    with pytest.raises(ValueError):
        native.rt_set_state("g", np.zeros(N + 3))
    assert len(fake.calls) == n_calls  # the library was not called
    native.rt_set_state("g", np.zeros(N, dtype=np.float32), n_H=[1.0] * N)  # host arrays are converted
    assert fake.calls[-1][4] == native.RT_MEM_HOST


def test_set_absorbers_and_rates(fake):
    native.rt_set_absorbers("g", np.zeros(N), np.zeros(N))
    assert fake.calls[-1][3] == native.RT_MEM_HOST
    with pytest.raises(ValueError):
        native.rt_set_absorbers("g", np.zeros(N), np.zeros(N - 1))
    with pytest.raises(ValueError):
        native.rt_set_absorbers("g", np.zeros(N), FakeCudaTensor(N))
    # device rates in the grid's precision: float32 or float64, one dtype for both
    native.rt_set_rates("g", FakeCudaTensor(N, "torch.float32"), FakeCudaTensor(N, "torch.float32", ptr=0x9000))
    assert fake.calls[-1] == ("rates", 0x7000, 0x9000, native.RT_DTYPE_F32, native.RT_MEM_DEVICE)
    native.rt_set_rates("g", FakeCudaTensor(N), FakeCudaTensor(N))
    assert fake.calls[-1][3] == native.RT_DTYPE_F64
    with pytest.raises(TypeError):
        native.rt_set_rates("g", FakeCudaTensor(N, "torch.float32"), FakeCudaTensor(N))
    with pytest.raises(ValueError):
        native.rt_set_rates("g", FakeCudaTensor(N + 1), FakeCudaTensor(N + 1))
    native.rt_set_rates("g", np.ones(N, dtype=np.float32), np.ones(N))  # host: sent as FP64
    assert fake.calls[-1][3] == native.RT_DTYPE_F64 and fake.calls[-1][4] == native.RT_MEM_HOST


def test_noalloc_grid_arrays(fake):
    params = native.trace_params()
    f32 = dict(dtype="torch.float32")

    def arrays(**over):
        a = dict(n_HI=FakeCudaTensor(N, ptr=1, **f32), n_H=FakeCudaTensor(N, ptr=2), x_HI=FakeCudaTensor(N, ptr=3),
                 kph=FakeCudaTensor(N, ptr=4, **f32), gamma=FakeCudaTensor(N, ptr=5, **f32))
        a.update(over)
        return a

    src = dict(pos_cm=np.zeros((2, 3)), ndot=[1e48, 1e48], e_ph_eV=[13.6, 13.6], sigma_cm2=[6.3e-18, 6.3e-18])
    native.rt_trace_noalloc((4, 5, 6), 1.0, **arrays(), **src, params=params)
    assert fake.calls[-1] == ("noalloc", 1, 2, 3, 4, 5, 2)
    with pytest.raises(TypeError):  # n_HI must be float32
        native.rt_trace_noalloc((4, 5, 6), 1.0, **arrays(n_HI=FakeCudaTensor(N)), **src, params=params)
    with pytest.raises(ValueError):  # host arrays are not accepted here
        native.rt_trace_noalloc((4, 5, 6), 1.0, **arrays(x_HI=np.zeros(N)), **src, params=params)
    with pytest.raises(ValueError):
        native.rt_trace_noalloc((4, 5, 6), 1.0, **arrays(kph=FakeCudaTensor(N - 1, **f32)), **src, params=params)
    with pytest.raises(ValueError):
        native.rt_trace_noalloc((4, 5, 6), 1.0, **arrays(), **dict(src, ndot=[1e48]), params=params)


def test_read_backs_check_the_cell_count(fake):
    for call in (lambda: native.rt_get_rates("g", N + 1), lambda: native.rt_get_ionised("g", N - 1),
                 lambda: native.rt_get_rates_typed("g", 2 * N, 1)):
        with pytest.raises(ValueError):
            call()
