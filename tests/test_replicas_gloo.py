"""Multi-replica host path of bench.py on the CPU: two gloo ranks (world size 2) reduce their timed
values with max_over_ranks, the only exchange of the replica benchmark (no data-path collective)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(tdist, values[rank], torch.device("cpu"))
        out.put((rank, got, bench.max_over_ranks(None, values[rank], None)))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("values", [(3.25, 7.5), (9.0, -1.0)])
def test_max_over_two_gloo_ranks(values):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in res) == [0, 1]
    for r, got, alone in res:
        assert got == max(values)          # every replica sees the slowest one
        assert alone == values[r]          # without a process group the value is its own
