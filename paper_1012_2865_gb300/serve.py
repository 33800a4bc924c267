"""Continuous-batching request loop for radiative-transfer solves.

A request is one grid (medium + sources) advanced by `nsteps` coupled steps
(rt_trace + rt_chem_update).  The server keeps the grids of all admitted
requests resident on the device in one rt_batch; every step advances all of
them with one persistent trace launch and one update launch.  Requests that
arrive while others run are admitted between steps when a slot is free and
the device has room for their grid (free HBM minus a reserve); finished
requests are read back to the host and leave the batch.  All computation
runs in librt_gb300.so; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import native, synth


def grid_bytes(ncell: int, precision: str) -> int:
    """Device bytes of one grid: n_H, x_HI, x_HII (FP64) + n_HI, k_ph, Gamma
    (FP64, or FP32 with n_HI as an FP32 pair)."""
    return ncell * (24 + (24 if precision == "fp64" else 16))


@dataclass
class Request:
    rid: int
    grid: dict
    nsteps: int
    arrival: float = 0.0      # seconds on the server clock
    admitted: float = -1.0
    finished: float = -1.0
    steps_done: int = 0
    slot: int = -1
    handle: object = None
    x_HI: np.ndarray = None
    kph: np.ndarray = None
    segments: int = 0
    meta: dict = field(default_factory=dict)
    factory: object = None    # builds `grid` at admission when it is None (a long stream)
    cells_hint: int = 0       # cells of that grid, for admission before it exists

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def cells(self) -> int:
        return int(np.prod(self.grid["dims"])) if self.grid is not None else int(self.cells_hint)


class Server:
    """`mem_info` (free device bytes), `mem_total` (the device's bytes) and
    `backend` (a module with the native.Grid and native.Batch classes) may be
    replaced, so that the scheduling can be exercised without a device."""

    def __init__(self, ctx, precision: str = "fp32_mixed", max_slots: int = 64,
                 reserve_bytes: int = 4 << 30, dt_s: float = 0.5 * synth.MYR_S, nsub: int = 10,
                 alpha_B: float = synth.ALPHA_B, params: dict = None, mem_info=None, backend=None,
                 mem_total=None):
        self.backend = backend if backend is not None else native
        self.ctx = ctx
        self.precision = precision
        self.max_slots = max_slots
        self.reserve = reserve_bytes
        self.dt_s, self.nsub, self.alpha_B = dt_s, nsub, alpha_B
        self.params = dict(synth.DEFAULT_PARAMS)
        if params:
            self.params.update(params)
        self.batch = self.backend.Batch(ctx)
        self.pending = collections.deque()
        self.active = {}
        self.done = []
        self.rejected = []
        self.failed = []
        self.cancelled = []
        self.steps = 0
        self.segments = 0
        self.oom_retries = 100  # admissions a request may retry after a failed allocation
        self._mem_info = mem_info
        self._mem_total = mem_total

    def free_bytes(self) -> int:
        if self._mem_info is not None:
            return self._mem_info()
        import torch
        return torch.cuda.mem_get_info()[0]

    def total_bytes(self) -> int:
        if self._mem_total is not None:
            return self._mem_total()
        import torch
        return torch.cuda.mem_get_info()[1]

    def submit(self, req: Request):
        self.pending.append(req)

    def admit(self, now: float) -> int:
        """Admit pending requests while a slot and device memory are free.
        A request waits while the memory is taken (by this server's grids or
        by other users of the device); one larger than the whole device minus
        the reserve can never be admitted and is rejected (kept in
        `rejected`) instead of holding up the queue."""
        n = 0
        while self.pending and len(self.active) < self.max_slots:
            req = self.pending[0]
            need = grid_bytes(req.cells, self.precision)
            if need > self.total_bytes() - self.reserve:
                self.pending.popleft()
                req.finished = now
                req.meta["rejected"] = f"needs {need} bytes; the device holds {self.total_bytes()}, " \
                                       f"{self.reserve} of them reserved"
                self.rejected.append(req)
                continue
            if self.free_bytes() - need < self.reserve:
                break
            self.pending.popleft()
            err = getattr(self.backend, "RtError", native.RtError)
            try:
                if req.grid is None and req.factory is not None:
                    req.grid = req.factory()
                req.handle = self.backend.Grid(self.ctx, req.grid, self.precision)
                req.slot = self.batch.add(req.handle)
            except err as e:
                if req.handle is not None:  # built, but the batch refused it
                    req.handle.close()
                    req.handle = None
                req.slot = -1
                tries = req.meta.get("oom_retries", 0)
                if getattr(e, "code", None) == native.RT_ERR_OOM and tries < self.oom_retries:
                    # memory taken by another user of the device since the
                    # check: the request waits at the head of the queue
                    req.meta["oom_retries"] = tries + 1
                    self.pending.appendleft(req)
                    break
                req.finished = now
                req.meta["error"] = f"admission: {e}"
                self.failed.append(req)
                continue
            req.admitted = now
            self.active[req.slot] = req
            n += 1
        return n

    def _retire(self, slot: int, now: float, bucket: list, why: str = None):
        req = self.active.pop(slot)
        req.finished = now
        if why is not None:
            req.meta["error"] = why
        self.batch.remove(slot)
        req.handle.close()
        req.handle = None
        if req.factory is not None:
            req.grid = None  # built on demand: let its medium go
        bucket.append(req)

    def _trace_all(self, now_fn):
        """The batch's trace.  When it fails, each request is traced alone to
        find the ones that fail by themselves; they leave with the error and
        the others are traced again together (a failed trace has not changed
        any state: the update has not run).  If the batch still fails, the
        error cannot be attributed and every active request fails with it."""
        err = getattr(self.backend, "RtError", native.RtError)
        try:
            self.batch.trace(sync=True, **self.params)
            return
        except err as e:
            first = str(e)
        for slot, req in list(self.active.items()):
            try:
                req.handle.trace(**self.params)
            except err as e:
                self._retire(slot, now_fn(), self.failed, str(e))
        if not self.active:
            return
        try:
            self.batch.trace(sync=True, **self.params)
        except err as e:
            for slot in list(self.active):
                self._retire(slot, now_fn(), self.failed, f"{e} (after: {first})")

    def cancel(self, rid: int, now: float = 0.0) -> bool:
        """Withdraw a request that is waiting or running (between steps)."""
        for req in list(self.pending):
            if req.rid == rid:
                self.pending.remove(req)
                req.finished = now
                self.cancelled.append(req)
                return True
        for slot, req in list(self.active.items()):
            if req.rid == rid:
                self._retire(slot, now, self.cancelled)
                return True
        return False

    def step(self, now_fn) -> int:
        """One coupled step of every active request; returns requests finished."""
        if not self.active:
            return 0
        self._trace_all(now_fn)
        if not self.active:
            return 0
        err = getattr(self.backend, "RtError", native.RtError)
        try:
            self.batch.chem(self.dt_s, self.nsub, self.alpha_B)
        except err as e:
            # one launch updates every grid: the error belongs to all of them
            for slot in list(self.active):
                self._retire(slot, now_fn(), self.failed, f"update: {e}")
            return 0
        self.steps += 1
        finished = []
        for slot, req in list(self.active.items()):
            try:
                b = self.batch.budget(slot)
            except err as e:
                self._retire(slot, now_fn(), self.failed, f"budget: {e}")
                continue
            req.segments += b["segments"]
            self.segments += b["segments"]
            req.steps_done += 1
            if req.steps_done >= req.nsteps:
                finished.append(slot)
        for slot in finished:
            req = self.active[slot]
            try:
                r = req.handle.rates()  # waits for the batch's update
            except err as e:
                self._retire(slot, now_fn(), self.failed, f"read-back: {e}")
                continue
            self.active.pop(slot)
            req.x_HI, req.kph = r["x_HI"], r["kph"]
            req.finished = now_fn()
            self.batch.remove(slot)
            req.handle.close()
            req.handle = None
            if req.factory is not None:
                req.grid = None  # built on demand: let its medium go
            self.done.append(req)
        return sum(1 for slot in finished if slot not in self.active)

    def run(self, requests: list, time_limit_s: float = None) -> dict:
        """Serve a stream: request.arrival is in seconds from the start.  With
        `time_limit_s` the loop stops at the first step boundary after it; the
        report then counts the requests that arrived and are still queued or
        in progress."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while todo or self.pending or self.active:
            t = now()
            while todo and todo[0].arrival <= t:
                self.submit(todo.popleft())
            self.admit(t)
            if self.active:
                self.step(now)
            elif self.pending:
                time.sleep(0.001)  # waiting for device memory held elsewhere
            elif todo:
                time.sleep(max(0.0, min(todo[0].arrival - now(), 0.01)))
            if time_limit_s is not None and now() > time_limit_s:
                break
        t = now()
        while todo and todo[0].arrival <= t:
            self.submit(todo.popleft())
        return self.report(t, not_arrived=len(todo))

    def report(self, wall_s: float, not_arrived: int = 0) -> dict:
        lat = np.array([r.latency for r in self.done]) if self.done else np.array([np.nan])
        return dict(completed=len(self.done), rejected=len(self.rejected), failed=len(self.failed),
                    cancelled=len(self.cancelled), queued=len(self.pending), in_progress=len(self.active),
                    not_arrived=not_arrived, wall_s=wall_s, steps=self.steps,
                    segments=self.segments,
                    segments_per_s=self.segments / wall_s if wall_s > 0 else 0.0,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    requests_per_s=len(self.done) / wall_s if wall_s > 0 else 0.0)

    def close(self):
        for req in self.active.values():
            if req.handle is not None:
                req.handle.close()
        self.active.clear()
        self.batch.close()


class MediumPool:
    """Request media cut from one pre-generated log-normal field.

    Each request takes an N^3 sub-cube at a seeded random offset of a 256^3
    field (P(k) ~ k^-3, sigma_ln = 1, mean 1e-2 cm^-3), so media of any size
    up to 256 are available at request rate without per-request FFTs.
    """

    def __init__(self, side: int = 256, seed: int = synth.BASE_SEED + 5):
        self.side = side
        self.field = synth.lognormal_density(side, seed=seed).reshape(side, side, side)

    def request(self, spec: dict, rid: int, lazy: bool = False) -> Request:
        """The request of one stream entry; with `lazy` its medium is cut at
        admission (a long stream then holds only the entries)."""
        if lazy:
            N = min(int(spec["N"]), self.side)
            return Request(rid=rid, grid=None, nsteps=int(spec["nsteps"]), arrival=float(spec["arrival_s"]),
                           factory=lambda: self.request(spec, rid).grid, cells_hint=N ** 3)
        rng = np.random.default_rng(spec["seed"])
        N = min(int(spec["N"]), self.side)
        o = rng.integers(0, self.side - N + 1, 3)
        n = np.ascontiguousarray(self.field[o[2]:o[2] + N, o[1]:o[1] + N, o[0]:o[0] + N]).reshape(-1)
        box = synth.box_cm(N)
        pos, ndot, e, sg = synth.random_sources((N, N, N), box / N, int(spec["nsrc"]), 1e47, 1e50, rng)
        g = synth._grid(N, box, n, 1.0, pos, ndot, e, sg)
        return Request(rid=rid, grid=g, nsteps=int(spec["nsteps"]), arrival=float(spec["arrival_s"]))


def run_alone(ctx, req: Request, precision: str, dt_s: float = 0.5 * synth.MYR_S, nsub: int = 10,
              alpha_B: float = synth.ALPHA_B, params: dict = None) -> tuple:
    """The same request on its own grid, one step after another (reference path)."""
    p = dict(synth.DEFAULT_PARAMS)
    if params:
        p.update(params)
    grid = native.Grid(ctx, req.grid, precision)
    segs = 0
    for _ in range(req.nsteps):
        segs += grid.trace(**p)["segments"]
        grid.chem(dt_s, nsub, alpha_B)
    r = grid.rates()
    grid.close()
    return r["x_HI"], r["kph"], segs


def serve_one_at_a_time(ctx, requests: list, precision: str, time_limit_s: float = None, **kw) -> dict:
    """The reference server, live: requests are served in arrival order, one at
    a time, each on its own grid (run_alone, no batching); a request starts
    when it has arrived and the previous one has finished, and its latency is
    its finish time minus its arrival time.  Stops before starting a request
    once `time_limit_s` has passed."""
    t0 = time.perf_counter()
    done = []
    for r in sorted(requests, key=lambda q: q.arrival):
        now = time.perf_counter() - t0
        if time_limit_s is not None and now > time_limit_s:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.admitted = time.perf_counter() - t0
        r.x_HI, r.kph, r.segments = run_alone(ctx, r, precision, **kw)
        r.finished = time.perf_counter() - t0
        done.append(r)
    lat = np.array([r.latency for r in done]) if done else np.array([np.nan])
    wall = time.perf_counter() - t0
    return dict(completed=len(done), wall_s=wall, p50_ms=float(np.percentile(lat, 50) * 1e3),
                p99_ms=float(np.percentile(lat, 99) * 1e3), service_s=[r.finished - r.admitted for r in done],
                rids=[r.rid for r in done], latency_ms=[1e3 * r.latency for r in done])
