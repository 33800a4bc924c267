"""The serving loop's scheduling on the host, with a stand-in for the device
library (no GPU): admission by free slots and free device memory, continuous
batching (requests that arrive while others run join between steps),
retirement after their own number of steps, latency accounting, and the
rejection of a request that can never fit instead of a stalled queue.
"""
import time
import types

import numpy as np

from paper_1012_2865_gb300 import serve


class FakeRtError(RuntimeError):
    def __init__(self, msg, code=3):
        super().__init__(msg)
        self.code = code


class FakeGrid:
    live = []
    made = []
    oom_left = 0  # the next constructions that fail as if the device's memory were gone

    def __init__(self, ctx, g, precision):
        if g.get("invalid"):
            raise FakeRtError("rt_add_sources: source 0 axis 0 outside the box", code=1)
        if FakeGrid.oom_left > 0:
            FakeGrid.oom_left -= 1
            raise FakeRtError("rt_create_grid: cudaMalloc: out of memory", code=2)
        self.ncell = int(np.prod(g["dims"]))
        self.precision = precision
        self.poison = g.get("poison", False)  # its trace fails, alone or in a batch
        self.created = time.perf_counter()
        FakeGrid.live.append(self)
        FakeGrid.made.append(self)

    def rates(self):
        return {"x_HI": np.zeros(self.ncell), "kph": np.ones(self.ncell)}

    def trace(self, **kw):
        if self.poison:
            raise FakeRtError("device status 6")
        return {"segments": self.ncell}

    def close(self):
        if self in FakeGrid.live:
            FakeGrid.live.remove(self)


class FakeBatch:
    step_s = 0.0

    def __init__(self, ctx):
        self.slots = {}
        self.sizes = []

    def add(self, grid):
        s = next(i for i in range(len(self.slots) + 1) if i not in self.slots)
        self.slots[s] = grid
        return s

    def remove(self, slot):
        del self.slots[slot]

    def trace(self, sync=True, **kw):
        if any(gr.poison for gr in self.slots.values()):
            raise FakeRtError("device status 6")
        self.sizes.append(len(self.slots))
        if FakeBatch.step_s:
            time.sleep(FakeBatch.step_s)

    def chem(self, dt_s, nsub, alpha_B):
        pass

    def budget(self, slot):
        return {"segments": self.slots[slot].ncell}

    def close(self):
        pass


BACKEND = types.SimpleNamespace(Grid=FakeGrid, Batch=FakeBatch, RtError=FakeRtError)


def _request(rid, N, nsteps, arrival=0.0, poison=False, invalid=False):
    g = {"dims": (N, N, N), "poison": poison, "invalid": invalid}
    return serve.Request(rid=rid, grid=g, nsteps=nsteps, arrival=arrival)


def _server(total_bytes, reserve, max_slots, precision="fp32_mixed", held=lambda: 0):
    """A server on a device of `total_bytes`, of which `held()` belongs to
    other users of the device."""
    def free():
        used = sum(serve.grid_bytes(gr.ncell, gr.precision) for gr in FakeGrid.live)
        return total_bytes - used - held()
    FakeGrid.live.clear()
    return serve.Server(None, precision, max_slots=max_slots, reserve_bytes=reserve, mem_info=free,
                        mem_total=lambda: total_bytes, backend=BACKEND)


def test_admission_by_slots_and_memory():
    FakeBatch.step_s = 0.0
    one = serve.grid_bytes(16 ** 3, "fp32_mixed")
    reqs = [_request(i, 16, nsteps=1 + i % 3) for i in range(9)]
    # memory for two grids above the reserve, three slots: memory binds
    srv = _server(total_bytes=1000 + 2 * one, reserve=1000, max_slots=3)
    rep = srv.run(reqs)
    assert rep["completed"] == 9 and rep["rejected"] == 0
    assert max(srv.batch.sizes) == 2
    for r in srv.done:
        assert r.steps_done == r.nsteps
        assert r.segments == r.nsteps * 16 ** 3
        assert r.admitted >= r.arrival and r.finished >= r.admitted and r.latency >= 0
    assert rep["segments"] == sum(r.nsteps for r in reqs) * 16 ** 3
    assert not FakeGrid.live  # every retired grid was released
    # plenty of memory, two slots: slots bind
    srv = _server(total_bytes=1 << 40, reserve=0, max_slots=2)
    srv.run([_request(i, 16, nsteps=2) for i in range(5)])
    assert max(srv.batch.sizes) == 2 and len(srv.done) == 5


def test_requests_join_while_others_run():
    FakeBatch.step_s = 0.004
    reqs = [_request(0, 20, nsteps=12, arrival=0.0), _request(1, 12, nsteps=3, arrival=0.015),
            _request(2, 24, nsteps=4, arrival=0.02)]
    srv = _server(total_bytes=1 << 40, reserve=0, max_slots=8)
    rep = srv.run(reqs)
    FakeBatch.step_s = 0.0
    assert rep["completed"] == 3
    done = {r.rid: r for r in srv.done}
    # the later requests were admitted while the first was still on the device ...
    assert done[1].admitted < done[0].finished and done[2].admitted < done[0].finished
    # ... and the short one left before it
    assert done[1].finished < done[0].finished
    assert max(srv.batch.sizes) >= 2
    assert rep["p99_ms"] >= rep["p50_ms"] > 0


def test_a_request_waits_for_memory_held_elsewhere():
    FakeBatch.step_s = 0.0
    one = serve.grid_bytes(16 ** 3, "fp32_mixed")
    t0 = time.perf_counter()
    # another user of the device holds all of it for the first 30 ms
    held = lambda: 4 * one if time.perf_counter() - t0 < 0.03 else 0  # noqa: E731
    srv = _server(total_bytes=4 * one, reserve=0, max_slots=4, held=held)
    srv.submit(_request(0, 16, nsteps=1))
    assert srv.admit(0.0) == 0 and len(srv.pending) == 1 and not srv.rejected
    FakeGrid.made.clear()
    rep = srv.run([_request(1, 16, nsteps=2, arrival=0.0)])
    assert rep["completed"] == 2 and rep["rejected"] == 0
    assert len(FakeGrid.made) == 2 and min(gr.created for gr in FakeGrid.made) >= t0 + 0.03


def test_a_request_that_never_fits_is_rejected():
    FakeBatch.step_s = 0.0
    small = serve.grid_bytes(16 ** 3, "fp64")
    reqs = [_request(0, 64, nsteps=1), _request(1, 16, nsteps=2), _request(2, 16, nsteps=1)]
    srv = _server(total_bytes=10 * small, reserve=0, max_slots=4, precision="fp64")
    rep = srv.run(reqs)
    assert rep["rejected"] == 1 and srv.rejected[0].rid == 0
    assert "rejected" in srv.rejected[0].meta
    assert rep["completed"] == 2 and sorted(r.rid for r in srv.done) == [1, 2]


def test_grid_bytes_counts_the_resident_fields():
    # n_H, x_HI, x_HII in FP64; n_HI, k_ph, Gamma in FP64 or (FP32 pair, FP32, FP32)
    assert serve.grid_bytes(1, "fp64") == 3 * 8 + 3 * 8
    assert serve.grid_bytes(1, "fp32_mixed") == 3 * 8 + 8 + 4 + 4


def test_a_failing_request_leaves_and_the_others_finish():
    FakeBatch.step_s = 0.0
    reqs = [_request(0, 16, nsteps=3), _request(1, 12, nsteps=2, poison=True), _request(2, 20, nsteps=4)]
    srv = _server(total_bytes=1 << 40, reserve=0, max_slots=8)
    rep = srv.run(reqs)
    assert rep["failed"] == 1 and srv.failed[0].rid == 1 and "status 6" in srv.failed[0].meta["error"]
    assert rep["completed"] == 2 and sorted(r.rid for r in srv.done) == [0, 2]
    assert all(r.steps_done == r.nsteps for r in srv.done)
    assert not FakeGrid.live


def test_cancel_waiting_and_running_requests():
    FakeBatch.step_s = 0.0
    one = serve.grid_bytes(16 ** 3, "fp32_mixed")
    srv = _server(total_bytes=one, reserve=0, max_slots=4)  # room for one grid at a time
    for i in range(3):
        srv.submit(_request(i, 16, nsteps=5))
    assert srv.admit(0.0) == 1
    srv.step(lambda: 0.1)
    assert srv.cancel(2, 0.2) and srv.cancel(0, 0.2)  # one waiting, one running
    assert not srv.cancel(7)
    assert [r.rid for r in srv.cancelled] == [2, 0]
    rep = srv.run([])
    assert rep["completed"] == 1 and srv.done[0].rid == 1 and rep["cancelled"] == 2
    assert not FakeGrid.live


def test_admission_failures_are_isolated():
    """A request whose grid the library refuses leaves with the error instead
    of ending the loop; one whose allocation fails (memory taken since the
    check) waits at the head of the queue and is admitted later."""
    FakeBatch.step_s = 0.0
    FakeGrid.oom_left = 2
    reqs = [_request(0, 16, nsteps=2), _request(1, 12, nsteps=1, invalid=True), _request(2, 20, nsteps=3)]
    srv = _server(total_bytes=1 << 40, reserve=0, max_slots=8)
    rep = srv.run(reqs)
    assert FakeGrid.oom_left == 0
    assert rep["failed"] == 1 and srv.failed[0].rid == 1 and "admission" in srv.failed[0].meta["error"]
    assert rep["completed"] == 2 and sorted(r.rid for r in srv.done) == [0, 2]
    assert srv.done[0].meta.get("oom_retries", 0) + srv.done[1].meta.get("oom_retries", 0) == 2
    assert not FakeGrid.live


def test_a_request_that_never_gets_its_memory_fails_after_its_retries():
    FakeBatch.step_s = 0.0
    FakeGrid.oom_left = 10 ** 6
    srv = _server(total_bytes=1 << 40, reserve=0, max_slots=8)
    srv.oom_retries = 5
    rep = srv.run([_request(0, 16, nsteps=1)])
    FakeGrid.oom_left = 0
    assert rep["failed"] == 1 and srv.failed[0].meta["oom_retries"] == 5
    assert "out of memory" in srv.failed[0].meta["error"]


def test_a_failing_update_fails_every_active_request():
    class BadChem(FakeBatch):
        def chem(self, dt_s, nsub, alpha_B):
            raise FakeRtError("rt_batch_chem: launch failed")
    FakeBatch.step_s = 0.0
    FakeGrid.live.clear()
    srv = serve.Server(None, "fp32_mixed", max_slots=4, reserve_bytes=0, mem_info=lambda: 1 << 40,
                       mem_total=lambda: 1 << 40,
                       backend=types.SimpleNamespace(Grid=FakeGrid, Batch=BadChem, RtError=FakeRtError))
    rep = srv.run([_request(0, 16, nsteps=2), _request(1, 16, nsteps=1)])
    assert rep["failed"] == 2 and rep["completed"] == 0
    assert all("update" in r.meta["error"] for r in srv.failed)
    assert not FakeGrid.live


def test_lazy_requests_and_a_time_limited_stream():
    """A long stream holds only its entries: a request's grid is built at
    admission and dropped when it leaves; a run cut at a time limit reports
    what arrived and is still queued or in progress."""
    FakeBatch.step_s = 0.003
    built = []

    def lazy(rid, N, nsteps, arrival):
        def make():
            built.append(rid)
            return {"dims": (N, N, N), "poison": False}
        return serve.Request(rid=rid, grid=None, nsteps=nsteps, arrival=arrival, factory=make, cells_hint=N ** 3)

    one = serve.grid_bytes(16 ** 3, "fp32_mixed")
    reqs = [lazy(i, 16, nsteps=4, arrival=0.002 * i) for i in range(40)] + [lazy(99, 16, 1, arrival=10.0)]
    srv = _server(total_bytes=3 * one, reserve=0, max_slots=8)
    rep = srv.run(reqs, time_limit_s=0.1)
    FakeBatch.step_s = 0.0
    assert rep["not_arrived"] == 1 and 99 not in built
    assert rep["completed"] + rep["queued"] + rep["in_progress"] == 40
    assert rep["completed"] > 0 and rep["queued"] > 0 and rep["in_progress"] <= 3
    assert sorted(built) == sorted([r.rid for r in srv.done] + [r.rid for r in srv.active.values()])
    assert all(r.grid is None for r in srv.done)
    assert max(srv.batch.sizes) <= 3  # memory for three grids
    srv.close()
