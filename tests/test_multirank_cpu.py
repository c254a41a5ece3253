"""The benchmark's multi-rank host logic on CPU (gloo, world size 2).

With N GPUs every rank parses its own text (weak scaling): the whole-job
figure is the units all ranks processed over the slowest rank's timed
region.  No collective touches the data path; the only ones are the barrier
and the two reductions checked here.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    ms = [3.0, 5.0][rank]
    units = [1000, 2500][rank]
    dist.barrier()
    got = bench.aggregate(ms, units, dist, torch.device("cpu"))
    text = W.dna_text(4096, seed=bench.rank_seed(1, rank))
    q.put((rank, got, bytes(text[:64])))
    dist.destroy_process_group()


def test_two_rank_aggregate_and_own_texts():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for _, got, _ in out:
        assert got == (5.0, 3500)                   # slowest rank's time, units summed
    assert out[0][2] != out[1][2]                   # each rank has its own input


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.5, 7) == (2.5, 7)
