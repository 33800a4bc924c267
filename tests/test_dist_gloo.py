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
