"""bench.py's multi-rank plumbing (replicas under torchrun) on CPU: two gloo
ranks agree on the barrier, the max of the step times (the job's ms/step) and
the sum of the particle-iterations/s. The data path has no collective: each
rank steps its own replica of the scene."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    d = bench.Dist()
    try:
        d.barrier()
        ms = [2.5, 3.25][rank]
        rate = [4.0e9, 3.0e9][rank]
        q.put((rank, d.ws, d.rank, d.max(ms), d.sum(rate)))
        d.barrier()
    finally:
        d.close()


def test_two_gloo_ranks_reduce_step_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, mx, sm in got:
        assert ws == 2 and r == rank
        assert mx == pytest.approx(3.25) and sm == pytest.approx(7.0e9)


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench

    d = bench.Dist()
    assert d.ws == 1 and d.pg is None
    assert d.max(1.5) == 1.5 and d.sum(2.0) == 2.0
    d.barrier()
    d.close()
