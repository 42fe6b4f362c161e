"""The multi-rank arithmetic of bench.py on world size 2 over gloo (CPU): whole-job throughput
is the DOF-updates of all ranks over the slowest rank's time (weak scaling, replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        red = bench.RankReducer(dist, "cpu")
        # rank r: its own replica with (r + 1) * 1000 DOFs per step, 4 steps, r-dependent time
        dofs = (rank + 1) * 1000.0
        ms = 10.0 + 5.0 * rank
        value, ms_max = bench.throughput(red, dofs, 4, ms)
        q.put((rank, value, ms_max, red.max(rank), red.sum(rank + 1)))
    finally:
        dist.destroy_process_group()


def test_throughput_over_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max, mx, sm in out:
        assert ms_max == 15.0                               # slowest rank
        assert value == pytest.approx((1000 + 2000) * 4 / 0.015)
        assert mx == 1 and sm == 3


def test_single_process_reducer_is_identity():
    import bench
    red = bench.RankReducer()
    assert red.max(2.5) == 2.5 and red.sum(3) == 3.0
    v, ms = bench.throughput(red, 100.0, 5, 20.0)
    assert ms == 20.0 and v == pytest.approx(100 * 5 / 0.02)
