"""Multi-rank host logic of the benchmark on CPU (two gloo ranks).

With N GPUs the benchmark runs one independent replica per rank: the
reported time is the slowest rank's, the work is summed over ranks, and the
timed region is bracketed by barriers.  These are exercised here without a
GPU, on the gloo backend, rendezvous on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier()
    t, n = bench.reduce_over_ranks(total_s=1.5 + rank, segments=1000 * (rank + 1))
    bench.barrier()
    q.put((rank, t, n, bench._dist()))
    dist.destroy_process_group()


def test_replicas_report_slowest_time_and_total_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, (r_env, w_env, _) in out:
        assert t == 2.5 and n == 3000  # max(1.5, 2.5); 1000 + 2000
        assert (r_env, w_env) == (rank, world)


def test_single_process_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(1.25, 7) == (1.25, 7)


def _shard_rank(rank, world, port, q):
    """One rank of a source-partitioned trace, the oracle standing in for the
    GPU tracer: trace the rank's sources, all-reduce rates and budget."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    from paper_1012_2865_gb300 import shard, synth
    g = synth.clumpy(N=20, nsrc=7, seed=21)
    sub, s0 = shard.shard_of(g, rank, world)
    o = oracle.trace(sub["dims"], sub["box_len_cm"], sub["n_H"], sub["x_HI"], sub["pos_cm"], sub["ndot"],
                     sub["e_ph_eV"], sub["sigma_cm2"], src_offset=s0, **synth.DEFAULT_PARAMS)
    k = torch.from_numpy(o["kph"].copy())
    gm = torch.from_numpy(o["gamma"].copy())
    f, i = shard.budget_vector(dict(emitted=o["budget"][0], absorbed=o["budget"][1], escaped=o["budget"][2],
                                    counts=o["counts"], hashes=o["hashes"], segments=o["segments"]))
    ft, it = torch.from_numpy(f), torch.from_numpy(i)
    for t in (k, gm, ft, it):
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    q.put((rank, k.numpy(), gm.numpy(), shard.budget_from_vector(ft.numpy(), it.numpy()), len(sub["ndot"])))
    dist.destroy_process_group()


def test_source_partitioned_trace_sums_to_the_whole():
    import numpy as np
    import oracle
    from paper_1012_2865_gb300 import synth
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.clumpy(N=20, nsrc=7, seed=21)
    full = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"], g["e_ph_eV"],
                        g["sigma_cm2"], **synth.DEFAULT_PARAMS)
    assert sum(t[4] for t in out) == 7 and all(t[4] > 0 for t in out)
    for _, k, gm, b, _ in out:  # every rank holds the whole trace's results
        np.testing.assert_array_equal(b["counts"], full["counts"])
        np.testing.assert_array_equal(b["hashes"], full["hashes"])
        assert b["segments"] == full["segments"]
        for j, key in enumerate(("emitted", "absorbed", "escaped")):
            assert abs(b[key] - full["budget"][j]) <= 1e-12 * full["budget"][0]
        np.testing.assert_allclose(k, full["kph"], rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(gm, full["gamma"], rtol=1e-12, atol=1e-300)


def _shard_fsl_rank(rank, world, port, q):
    """A source-partitioned trace with a finite speed of light: each rank keeps
    the packages in flight of its own sources from step to step."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    from paper_1012_2865_gb300 import shard, synth
    g = synth.clumpy(N=16, nsrc=5, seed=31)
    g["x_HI"] = np.full(16 ** 3, 0.02)
    sub, s0 = shard.shard_of(g, rank, world)
    light = 3.5 * g["box_len_cm"] / 16
    fl = oracle.Flight()
    steps = []
    for step in range(4):
        o = oracle.trace(sub["dims"], sub["box_len_cm"], sub["n_H"], sub["x_HI"], sub["pos_cm"], sub["ndot"],
                         sub["e_ph_eV"], sub["sigma_cm2"], src_offset=s0, flight=fl, light_cm=light,
                         **synth.DEFAULT_PARAMS)
        k = torch.from_numpy(o["kph"].copy())
        f, i = shard.budget_vector(dict(emitted=o["budget"][0], absorbed=o["budget"][1], escaped=o["budget"][2],
                                        resumed=o["resumed"], halted=o["halted"], counts=o["counts"],
                                        hashes=o["hashes"], segments=o["segments"]))
        ft, it = torch.from_numpy(f), torch.from_numpy(i)
        for t in (k, ft, it):
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
        steps.append((k.numpy(), shard.budget_from_vector(ft.numpy(), it.numpy())))
    q.put((rank, steps))
    dist.destroy_process_group()


def test_source_partitioned_trace_with_packages_in_flight():
    import numpy as np
    import oracle
    from paper_1012_2865_gb300 import synth
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_fsl_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.clumpy(N=16, nsrc=5, seed=31)
    g["x_HI"] = np.full(16 ** 3, 0.02)
    fl = oracle.Flight()
    for step in range(4):
        full = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], g["x_HI"], g["pos_cm"], g["ndot"],
                            g["e_ph_eV"], g["sigma_cm2"], flight=fl, light_cm=3.5 * g["box_len_cm"] / 16,
                            **synth.DEFAULT_PARAMS)
        total = full["budget"][0] + full["resumed"]
        for _, steps in out:
            k, b = steps[step]
            np.testing.assert_array_equal(b["counts"], full["counts"])
            np.testing.assert_array_equal(b["hashes"], full["hashes"])
            assert b["segments"] == full["segments"]
            for key, ref in (("emitted", full["budget"][0]), ("absorbed", full["budget"][1]),
                             ("escaped", full["budget"][2]), ("resumed", full["resumed"]), ("halted", full["halted"])):
                assert abs(b[key] - ref) <= 1e-12 * total, (step, key)
            np.testing.assert_allclose(k, full["kph"], rtol=1e-12, atol=1e-300)
    assert full["resumed"] > 0 and full["halted"] > 0


def test_source_ranges_partition_the_list():
    from paper_1012_2865_gb300 import shard
    for nsrc in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            got = [shard.source_range(nsrc, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == nsrc
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(b - a for a, b in got) - min(b - a for a, b in got) <= 1


class _OracleGrid:
    """Stands in for native.Grid on the host: the oracle traces the grid's
    sources (with their global numbering) and updates its state."""

    def __init__(self, ctx, g, precision):
        import numpy as np
        self.g = dict(g)
        self.h = self
        self.ncell = int(np.prod(g["dims"]))
        self.x = np.asarray(g["x_HI"], dtype=np.float64).copy()
        self.z = np.asarray(g.get("x_HII", 1.0 - self.x), dtype=np.float64).copy()
        self.off = 0
        self.kph = self.gamma = None

    def add(self, pos, ndot, e, sg):
        self.g.update(pos_cm=pos, ndot=ndot, e_ph_eV=e, sigma_cm2=sg)

    def trace(self, **params):
        import oracle
        g = self.g
        o = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], self.x, g["pos_cm"], g["ndot"], g["e_ph_eV"],
                         g["sigma_cm2"], src_offset=self.off, **params)
        self.kph, self.gamma = o["kph"], o["gamma"]
        return dict(emitted=o["budget"][0], absorbed=o["budget"][1], escaped=o["budget"][2], counts=o["counts"],
                    hashes=o["hashes"], segments=o["segments"])

    def chem(self, dt_s, nsub, alpha_B):
        import oracle
        self.x, self.z = oracle.chem(self.g["n_H"], self.x, self.z, self.kph, dt_s, nsub, alpha_B)

    def close(self):
        pass


def _oracle_backend():
    import types
    import numpy as np

    def set_rates(h, k, g):
        h.kph, h.gamma = np.asarray(k, dtype=np.float64), np.asarray(g, dtype=np.float64)
    return types.SimpleNamespace(
        Grid=_OracleGrid, rt_set_source_offset=lambda h, s0: setattr(h, "off", s0),
        rt_add_sources=lambda h, pos, ndot, e, sg: h.add(pos, ndot, e, sg),
        rt_get_rates=lambda h, n, dt, where: {"kph": h.kph.copy(), "gamma": h.gamma.copy()},
        rt_set_rates=set_rates)


def _shard_step_rank(rank, world, port, q):
    """ShardGrid.step on gloo: each rank traces its share of the sources, the
    rates and budgets are summed over the ranks, every rank installs the sums
    and updates its (identical) state."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1012_2865_gb300 import shard, synth
    g = synth.clumpy(N=16, nsrc=6, seed=41)
    sg = shard.ShardGrid(None, g, "fp64", rank, world, backend=_oracle_backend())
    out = []
    for _ in range(2):
        b = sg.step(0.5 * synth.MYR_S, 10, synth.ALPHA_B, **synth.DEFAULT_PARAMS)
        out.append((b, sg.grid.kph.copy(), sg.grid.x.copy()))
    q.put((rank, out))
    dist.destroy_process_group()


def test_shard_grid_step_exchanges_once_per_trace():
    """Two coupled steps of a source-partitioned grid through ShardGrid.step
    (the path a multi-GPU run takes, here on gloo with the oracle as each
    rank's tracer) equal the same steps of the whole grid on one process."""
    import numpy as np
    import oracle
    from paper_1012_2865_gb300 import synth
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_step_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.clumpy(N=16, nsrc=6, seed=41)
    x, z = np.asarray(g["x_HI"], dtype=np.float64), np.asarray(g["x_HII"], dtype=np.float64)
    for step in range(2):
        full = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], x, g["pos_cm"], g["ndot"], g["e_ph_eV"],
                            g["sigma_cm2"], **synth.DEFAULT_PARAMS)
        x, z = oracle.chem(g["n_H"], x, z, full["kph"], 0.5 * synth.MYR_S, 10, synth.ALPHA_B)
        for _, steps in out:
            b, k, xr = steps[step]
            np.testing.assert_array_equal(b["counts"], full["counts"])
            np.testing.assert_array_equal(b["hashes"], full["hashes"])
            assert b["segments"] == full["segments"]
            for j, key in enumerate(("emitted", "absorbed", "escaped")):
                assert abs(b[key] - full["budget"][j]) <= 1e-12 * full["budget"][0]
            np.testing.assert_allclose(k, full["kph"], rtol=1e-12, atol=1e-300)
            np.testing.assert_allclose(xr, x, rtol=1e-12, atol=1e-15)
