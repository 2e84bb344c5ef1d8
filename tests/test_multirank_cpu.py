"""Multi-rank bench logic on CPU (gloo, world size 2): each rank runs its own replica, the job
time is the slowest rank's time and the value counts every rank's pairs (weak scaling)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    job_ms, value = bench.aggregate_ranks(local_ms, pairs_per_step=1000, steps=4, ws=ws, device="cpu")
    q.put((rank, job_ms, value))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_max_over_ranks_and_total_pairs(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, value in res:
        assert job_ms == pytest.approx(100.0 * ws)
        assert value == pytest.approx(ws * 1000 * 4 / (job_ms * 1e-3))


def test_single_rank_needs_no_process_group():
    import bench

    job_ms, value = bench.aggregate_ranks(250.0, 10, 5, 1)
    assert job_ms == 250.0 and value == pytest.approx(10 * 5 / 0.25)
