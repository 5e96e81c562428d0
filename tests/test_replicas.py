"""The multi-GPU path of the benchmark is independent replicas (the sampler
does not shard): rank 0's splitting and grid are broadcast, each replica
draws its own noise, and the whole-job value is every replica's samples
over the slowest replica's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        dev = torch.device("cpu")
        xi, M = bench.replica_plan(0.5 + 0.01 * rank, 256 + 6 * rank, dev)
        t = bench.replica_time(10.0 + 5.0 * rank, dev)
        dist.barrier()
        q.put((rank, xi, M, t, bench.replica_seed(rank), bench.replica_value(ws, 1000, 4, t)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_plan_and_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = root + (os.pathsep + old if old else "")
    try:
        for p in procs:
            p.start()
        res = sorted(q.get(timeout=120) for _ in range(ws))
    finally:
        os.environ["PYTHONPATH"] = old
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, xi, M, t, seed, value in res:
        assert (xi, M) == (0.5, 256)          # rank 0's choice everywhere
        assert t == 15.0                      # the slower rank's time
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)
    assert res[0][4] != res[1][4]             # independent noise per replica
