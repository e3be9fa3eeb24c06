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


def _batch_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_1608_04721_gb300 import scenes

    d = bench.Dist()
    try:
        sizes = [c.n for c in scenes.config_batch_256()]
        mine = bench.partition_scenes(sizes, d.ws)[d.rank]
        n_mine = sum(sizes[k] for k in mine)
        # the job's particles and ms/step as the batch workload reduces them
        q.put((rank, mine, n_mine, d.sum(n_mine), d.max(1.0 + rank)))
    finally:
        d.close()


def test_batch_scenes_split_over_two_gloo_ranks():
    """bench.py --workload batch_256 under two ranks: each rank steps its own
    whole scenes (particle-balanced), the two shares are disjoint and cover
    all 256 scenes, and the job's particle count and step time are the sum
    and the max over ranks."""
    from paper_1608_04721_gb300 import scenes

    sizes = [c.n for c in scenes.config_batch_256()]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a, na, tot_a, mx_a), (_, b, nb, tot_b, mx_b) = got
    assert not set(a) & set(b) and sorted(a + b) == list(range(256))
    assert tot_a == tot_b == sum(sizes) and mx_a == mx_b == 2.0
    assert abs(na - nb) <= max(sizes)


def test_partition_is_balanced_and_deterministic():
    import bench

    sizes = [5, 9, 1, 7, 3, 3, 8]
    parts = bench.partition_scenes(sizes, 3)
    assert parts == bench.partition_scenes(sizes, 3)
    assert sorted(k for p in parts for k in p) == list(range(len(sizes)))
    loads = [sum(sizes[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert bench.partition_scenes(sizes, 1) == [list(range(len(sizes)))]
