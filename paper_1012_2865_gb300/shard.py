"""One grid traced by several ranks, each holding a share of its sources.

The trace is linear in the sources: k_ph, Gamma, the photon budget, the
packages created per level (and their checksum) and the segment count of the
whole source list are the sums over any partition of it.  So each rank keeps
the full medium, traces its contiguous range of the sources (with that
range's global source numbering, for the checksum), and the ranks sum the
rates and the budget (one all-reduce each); every rank then holds the rates
of the whole trace and runs the same ionisation update, so the ranks' states
stay identical.  The exchange is the only communication per step.

`shard_trace` runs one rank's share and returns its partial results;
`allreduce` sums the partial rates (in place) and budgets over the ranks of a
`torch.distributed` process group -- NCCL with the rates as CUDA tensors, or
gloo with host tensors -- and `install` writes the sums back into the grid.
`ShardGrid.step` is one coupled step of the whole grid on one rank: its share
of the trace, the exchange, the installation and the (replicated) update.
With a finite speed of light the packages in flight belong to the sources
that emitted them, so each rank keeps its own between steps: `ShardGrid`
holds a rank's grid across steps, and the budget sums carry the photons
resumed and halted.
"""
from __future__ import annotations

import numpy as np

from . import native

BUDGET_KEYS = ("emitted", "absorbed", "escaped", "resumed", "halted")


def source_range(nsrc: int, rank: int, world: int) -> tuple:
    """Contiguous share [s0, s1) of nsrc sources for `rank` of `world`."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    return nsrc * rank // world, nsrc * (rank + 1) // world


def shard_of(g: dict, rank: int, world: int) -> tuple:
    """The grid description restricted to this rank's sources, and s0."""
    s0, s1 = source_range(len(g["ndot"]), rank, world)
    sub = dict(g)
    for k in ("pos_cm", "ndot", "e_ph_eV", "sigma_cm2"):
        sub[k] = np.asarray(g[k])[s0:s1]
    return sub, s0


def budget_vector(b: dict) -> tuple:
    """(FP64 sums, int64 counters) of a budget, in a fixed order for an
    all-reduce; the checksums wrap modulo 2^64 as int64 sums do."""
    f = np.array([b.get(k, 0.0) for k in BUDGET_KEYS], dtype=np.float64)
    i = np.concatenate([np.asarray(b["counts"], dtype=np.uint64), np.asarray(b["hashes"], dtype=np.uint64),
                        np.array([b["segments"]], dtype=np.uint64)]).view(np.int64)
    return f, i


def budget_from_vector(f, i) -> dict:
    u = np.asarray(i, dtype=np.int64).view(np.uint64)
    n = (len(u) - 1) // 2
    out = {k: float(v) for k, v in zip(BUDGET_KEYS, np.asarray(f, dtype=np.float64))}
    out.update(counts=u[:n].copy(), hashes=u[n:2 * n].copy(), segments=int(u[2 * n]))
    return out


def allreduce(kph, gamma, budget: dict, group=None) -> dict:
    """Sum k_ph and Gamma (torch tensors, summed in place) and the photon
    budget over the ranks of `group` (one exchange per trace); returns the
    whole trace's budget.  The budget travels on the rates' device."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return budget  # a single process holds the whole trace
    f, i = budget_vector(budget)
    ft = torch.from_numpy(f).to(kph.device)
    it = torch.from_numpy(i).to(kph.device)
    for t in (kph, gamma, ft, it):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return budget_from_vector(ft.cpu().numpy(), it.cpu().numpy())


def shard_trace(ctx, g: dict, precision: str, rank: int, world: int, where: str = "device", **params):
    """Trace this rank's sources on a grid holding the whole medium.

    Returns (grid, budget, kph, gamma): the partial budget and rates, the
    rates as CUDA tensors (where='device') or numpy arrays in the grid's
    precision."""
    sub, s0 = shard_of(g, rank, world)
    grid = native.Grid(ctx, dict(sub, ndot=[]), precision)  # sources added below, after the offset
    native.rt_set_source_offset(grid.h, s0)
    if len(sub["ndot"]):
        native.rt_add_sources(grid.h, sub["pos_cm"], sub["ndot"], sub["e_ph_eV"], sub["sigma_cm2"])
    b = grid.trace(**params)
    dt = native.RT_DTYPE_F64 if precision == "fp64" else native.RT_DTYPE_F32
    r = native.rt_get_rates(grid.h, grid.ncell, dt, where)
    return grid, b, r["kph"], r["gamma"]


class ShardGrid:
    """One rank's share of the sources on a grid that lives across steps.

    trace() returns the rank's partial (budget, kph, gamma); after the
    all-reduce, install() writes the sums into the grid and chem() advances
    the (identical on every rank) state."""

    def __init__(self, ctx, g: dict, precision: str, rank: int, world: int, backend=None):
        # `backend` (the native module by default) may be replaced by a
        # stand-in with the same calls, so the exchange can be exercised
        # without a device
        self.lib = backend if backend is not None else native
        sub, self.s0 = shard_of(g, rank, world)
        self.precision = precision
        self.nsrc = len(sub["ndot"])
        self.grid = self.lib.Grid(ctx, dict(sub, ndot=[]), precision)
        self.lib.rt_set_source_offset(self.grid.h, self.s0)
        if self.nsrc:
            self.lib.rt_add_sources(self.grid.h, sub["pos_cm"], sub["ndot"], sub["e_ph_eV"], sub["sigma_cm2"])

    def set_source_rates(self, ndot_all):
        """Rates of every source of the whole list; this rank takes its range."""
        if self.nsrc:
            self.grid.set_source_rates(np.asarray(ndot_all)[self.s0:self.s0 + self.nsrc])

    def trace(self, where: str = "device", **params):
        b = self.grid.trace(**params)
        dt = native.RT_DTYPE_F64 if self.precision == "fp64" else native.RT_DTYPE_F32
        r = self.lib.rt_get_rates(self.grid.h, self.grid.ncell, dt, where)
        return b, r["kph"], r["gamma"]

    def install(self, kph, gamma):
        self.lib.rt_set_rates(self.grid.h, kph, gamma)

    def step(self, dt_s: float, nsub: int, alpha_B: float, group=None, **params) -> dict:
        """One coupled step of the whole grid on this rank: trace this rank's
        sources, sum the rates and budgets over the ranks (NCCL: the rates stay
        CUDA tensors; gloo: host tensors), install the sums, update.  Returns
        the whole trace's budget."""
        import torch
        import torch.distributed as dist
        on_device = not dist.is_initialized() or dist.get_backend(group) == "nccl"
        b, kph, gamma = self.trace(where="device" if on_device else "host", **params)
        if not on_device:
            kph, gamma = torch.from_numpy(np.asarray(kph)), torch.from_numpy(np.asarray(gamma))
        total = allreduce(kph, gamma, b, group)
        self.install(kph if on_device else kph.numpy(), gamma if on_device else gamma.numpy())
        self.chem(dt_s, nsub, alpha_B)
        return total

    def chem(self, dt_s, nsub, alpha_B):
        self.grid.chem(dt_s, nsub, alpha_B)

    def close(self):
        self.grid.close()


def install(grid, kph, gamma):
    """Write the summed rates into the grid (before rt_chem_update)."""
    native.rt_set_rates(grid.h, kph, gamma)
