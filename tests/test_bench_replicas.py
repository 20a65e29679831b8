"""The benchmark's multi-GPU mode runs independent replicas (one per rank, no data-path collective):
the job's time is the slowest rank's and its solves all ranks'.  Checked with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 10 + 5 r ms on the device and 20 - r ms end to end, 40 solves each
        res = bench.replica_totals(10.0 + 5.0 * rank, 20.0 - rank, 40, world)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_solves():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(out.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert got[r] == (15.0, 20.0, 80)


def test_one_rank_is_its_own_total():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(12.5, 13.0, 40, 1) == (12.5, 13.0, 40)
