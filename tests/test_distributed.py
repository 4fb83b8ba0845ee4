"""The N > 1 path of bench.py (replicas, no data-path collective) on the CPU:
two gloo ranks check the max-over-ranks timing and the summed work that the
whole-job throughput is built from."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    import bench
    ws, r, local = bench.dist_setup()
    t_max = bench.barrier_max(1.0 + rank, ws)          # each replica's elapsed time
    flops = bench.barrier_sum(10.0 * (rank + 1), ws)   # each replica's work
    bench.barrier(ws)
    q.put((r, ws, t_max, flops, flops / t_max))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, t_max, flops, value in out:
        assert ws == 2
        assert t_max == 2.0            # the slower replica sets the time
        assert flops == 30.0           # work of both replicas
        assert value == 15.0           # whole-job throughput
